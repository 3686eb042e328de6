// te_server.cu - serving engine: continuous batching of many small Top-K
// solves on one GPU.
//
// Host side.  A first-fit pool allocator hands out device memory from one
// allocation; requests wait in submission order until a slot and enough pool
// memory are free; admission builds the solve's SELL layout and state on the
// device and runs its start-vector pass; every engine step then advances all
// resident solves by one Lanczos step with the batched kernels (one launch per
// phase, replayed as one captured graph that reads a device table of the
// resident solves).  A solve that completes its m steps gets its Jacobi and
// Ritz kernels in the same step; its work memory is freed at the next step and
// its Ritz vectors stay in the pool until the client polls them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "te_internal.h"
#include "topk_eigs.h"

using namespace te;

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

te_status srv_fail(te_status s, const std::string& m) {
  set_last_error(m);
  return s;
}
te_status srv_cuda(cudaError_t e, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                 ")");
  return e == cudaErrorMemoryAllocation ? TE_ERR_OUT_OF_MEMORY : TE_ERR_CUDA;
}
#define SRV_CK(call, what)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return srv_cuda(e_, what);   \
  } while (0)

// First-fit allocator over one device allocation (offsets, 256-byte aligned);
// freed blocks merge with free neighbours.
class Pool {
 public:
  char* base = nullptr;
  size_t size = 0, used = 0, peak = 0;
  cudaError_t init(size_t bytes) {
    size = al256(bytes);
    cudaError_t e = cudaMalloc(&base, size);
    if (e == cudaSuccess) free_[0] = size;
    return e;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al256(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t roff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[roff] = rest;
      used += bytes;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(std::max<size_t>(bytes, 1));
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  ~Pool() {
    if (base) cudaFree(base);
  }

 private:
  std::map<size_t, size_t> free_;
};

// pending -> admitted (layout built, columns being checked on the device) ->
// running (resident in the batch) -> finished
// pending -> admitted -> running -> finishing (Jacobi, Ritz vectors on the
// finishing stream) -> finished
enum ReqState {
  REQ_PENDING = 0,
  REQ_RUNNING = 1,
  REQ_FINISHED = 2,
  REQ_ADMITTED = 3,
  REQ_FINISHING = 4
};

struct Request {
  int64_t ticket = 0;
  int64_t n = 0, nnz = 0, n_pad = 0;
  // the caller's CSR (borrowed: it stays valid until the request is done)
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const void* vals = nullptr;  // binary64 or binary32, as given
  size_t val_bytes = 0;
  int in_type = TE_F32, vk = TE_F32;
  int K = 0, m = 0, ncta = 1;
  uint64_t seed = 0;
  int state = REQ_PENDING, status = 0, slot = -1, step = 0;
  size_t work_off = 0, work_bytes = 0, res_off = 0, res_bytes = 0;
  BatchSlot desc{};
  std::vector<double> theta, resid;
  // the SpMV layout, built by an analysis thread after submission (with the
  // layout candidate `cand` of the autotuner's list)
  SellHost layout;
  int cand = 0;
  // its sizes (from the host build, or from the device build, which fills
  // the staged arrays directly and leaves `layout` empty)
  size_t ls_slices = 0, ls_lanes = 0, ls_lrows = 0;
  int64_t ls_entries = 0, ls_pieces = 0;
  // the CSR and the layout copied to the device staging area by the analysis
  // thread (stage_bytes = 0: not staged; admission copies from the host)
  int64_t seq = 0;  // submission order
  size_t stage_off = 0, stage_bytes = 0;
  std::atomic<int> analysed{0};
};

// Host threads that build the SpMV layouts of submitted requests while the
// engine runs, so that admission only allocates, copies and launches.
// An analysis thread's pinned bounce buffer: a request's arrays are copied
// into it by the CPU and go to the device in one DMA.  (Copies straight from
// pageable memory issued by several threads at once ran at ≈ 5 GB/s per
// thread, and worse the more threads issued them.)
constexpr size_t BOUNCE_MAX = (size_t)256 << 20;  // larger requests copy from pageable memory
struct Bounce {
  char* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t b) {
    if (b <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(b + b / 2, (size_t)64 << 20);
    if (cudaHostAlloc(reinterpret_cast<void**>(&p), want, cudaHostAllocDefault) != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
      return false;
    }
    cap = want;
    return true;
  }
  ~Bounce() {
    if (p) cudaFreeHost(p);
  }
};

class AnalysisPool {
 public:
  // fn builds a request's layout (on an analysis thread, device `dev`
  // current, with a stream and a bounce buffer of its own)
  void start(unsigned nthreads, int dev,
             std::function<void(Request*, cudaStream_t, Bounce*)> fn) {
    fn_ = std::move(fn);
    dev_ = dev;
    for (unsigned t = 0; t < nthreads; ++t) th_.emplace_back([this] { run(); });
  }
  void post(Request* R) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      q_.push_back(R);
    }
    cv_.notify_one();
  }
  // block until R's layout is built
  void wait(Request* R) {
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [R] { return R->analysed.load(std::memory_order_acquire) != 0; });
  }
  void stop() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
    th_.clear();
  }
  ~AnalysisPool() { stop(); }

 private:
  void run() {
    cudaSetDevice(dev_);
    cudaStream_t ts = nullptr;
    cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    Bounce bounce;
    for (;;) {
      Request* R = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [this] { return stop_ || !q_.empty(); });
        if (stop_) break;
        R = q_.front();
        q_.pop_front();
      }
      fn_(R, ts, &bounce);
      {
        std::lock_guard<std::mutex> lk(mu_);
        R->analysed.store(1, std::memory_order_release);
      }
      done_.notify_all();
    }
    if (ts) {
      cudaStreamSynchronize(ts);
      cudaStreamDestroy(ts);
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  std::deque<Request*> q_;
  bool stop_ = false;
  int dev_ = 0;
  std::function<void(Request*, cudaStream_t, Bounce*)> fn_;
};

struct SlotResult {  // pinned, written by the finishing copies
  double theta[MAX_M];
  double resid[MAX_M];
  int hdr[4];  // restart_flag, restarts, status, sweeps (as in LzState)
  int bad_cols;  // admission: a column index outside [0, n)
  int pad_;
};

int64_t pad_rows(int64_t n) { return (n + TILE_R - 1) / TILE_R * TILE_R; }

// pass CTAs of a solve: a function of its size alone
int ctas_for(int64_t n_pad) {
  const int64_t tiles = n_pad / TILE_R;
  int64_t c = (tiles + 3) / 4;
  if (c < 1) c = 1;
  if (c > SRV_MAX_CTAS) c = SRV_MAX_CTAS;
  return (int)c;
}

}  // namespace

struct te_server {
  int max_slots = 0, max_m = 0, use_graph = 1, num_sms = 0;
  int spmv_blocks = 0, fin_blocks = 0;  // persistent grids of the batched SpMV and finaliser
  // admissions run on their own stream, beside the engine step: a copy from
  // pageable host memory first waits for the work already queued on its
  // stream, which then is only the earlier admissions
  cudaStream_t as = nullptr;
  cudaEvent_t ev_admit = nullptr;
  bool admit_pending = false;
  cudaStream_t s = nullptr, ps = nullptr;  // engine stream, poll stream
  Pool pool;
  PassLaunch Lpass{}, Lritz{}, Lsto{};
  BatchTable* table_h = nullptr;
  BatchTable* table_d = nullptr;
  SlotResult* res_h = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  int64_t next_ticket = 1;
  std::map<int64_t, Request*> reqs;
  std::deque<Request*> pending;
  std::vector<Request*> slots;
  std::vector<std::pair<size_t, size_t>> deferred;  // pool blocks to free after the next sync
  // solves that completed their m steps: their Jacobi and Ritz kernels run on
  // finishing streams, beside the following engine steps (round robin over
  // SRV_FIN_STREAMS streams, so that the Jacobi kernels of solves finishing
  // close together run at the same time on different SMs), and they are
  // retired when their batch's event has completed
  static constexpr int SRV_FIN_STREAMS = 8;
  cudaStream_t fs[SRV_FIN_STREAMS] = {};
  int fs_next = 0;
  cudaEvent_t ev_step = nullptr;
  struct FinishBatch {
    cudaEvent_t ev;
    std::vector<int> slots;
  };
  std::deque<FinishBatch> batches;
  std::vector<cudaEvent_t> ev_free;
  std::deque<int64_t> completed;                    // finished tickets not yet reported
  // per request class (value type, log2 n, log2 mean row length): the
  // autotuner's layout candidate, tuned on the class's first request
  bool autotune = false;
  int dev = 0;
  // device staging area: analysis threads copy each request's CSR and layout
  // there in submission order (first-fit, freed after its admission), so that
  // admission issues no copy from pageable host memory
  Pool stage;
  std::mutex stage_mu;
  std::condition_variable stage_cv;
  int64_t next_seq = 0, stage_turn = 0;
  bool stopping = false;
  std::mutex tune_mu;
  std::condition_variable tune_cv;
  std::map<int, int> tuned;
  std::set<int> tuning;
  double t_wait = 0, t_admit = 0, t_launch = 0, t_submit = 0;  // host seconds, cumulative
  double t_poll_copy = 0, t_poll_free = 0;  // polls: the Ritz vectors' copy, the request's release
  // analysis threads (nanoseconds, summed over threads): layout builds, the
  // gathers into the bounce buffers, the DMAs into the staging area, waits
  // for the staging turn or space; requests analysed
  std::atomic<int64_t> a_layout_ns{0}, a_gather_ns{0}, a_stage_ns{0}, a_wait_ns{0}, a_count{0};
  int64_t engine_steps = 0, resident_steps = 0;  // steps launched, solves they advanced
  AnalysisPool analysis;
};

namespace {

int request_class(const Request* R) {
  int ln = 0, ld = 0;
  while (ln < 40 && ((int64_t)1 << (ln + 1)) <= R->n) ++ln;
  const int64_t deg = R->n > 0 ? R->nnz / R->n : 0;
  while (ld < 20 && ((int64_t)1 << (ld + 1)) <= deg) ++ld;
  return (R->vk * 64 + ln) * 32 + ld;
}

// Time the autotuner's layout candidates on R's matrix (its own stream and
// temporary device memory, beside the engine); -1 when the matrix cannot be
// tuned (a column index outside [0, n), or a CUDA error).
int tune_request(const Request* R) {
  cudaStream_t ts = nullptr;
  if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) return -1;
  const size_t b_rp = al256((size_t)(R->n + 1) * 8), b_ci = al256((size_t)R->nnz * 4 + 4),
               b_v = al256(R->val_bytes + 8);
  char* b = nullptr;
  int best = -1;
  cudaError_t e = dev_alloc(&b, b_rp + b_ci + b_v + 256);
  if (e == cudaSuccess) {
    int* flag = reinterpret_cast<int*>(b + b_rp + b_ci + b_v);
    e = cudaMemcpyAsync(b, R->rp, (size_t)(R->n + 1) * 8, cudaMemcpyHostToDevice, ts);
    if (e == cudaSuccess && R->nnz)
      e = cudaMemcpyAsync(b + b_rp, R->ci, (size_t)R->nnz * 4, cudaMemcpyHostToDevice, ts);
    if (e == cudaSuccess && R->nnz)
      e = cudaMemcpyAsync(b + b_rp + b_ci, R->vals, R->val_bytes, cudaMemcpyHostToDevice, ts);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), ts);
    if (e == cudaSuccess)
      e = launch_validate_cols(reinterpret_cast<const int32_t*>(b + b_rp), R->nnz, R->n, flag, ts);
    int hflag = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ts);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
    int c = 0;
    if (e == cudaSuccess && !hflag &&
        autotune_layout(PREC_FDF, R->vk, R->in_type, R->rp, reinterpret_cast<const int64_t*>(b),
                        reinterpret_cast<const int32_t*>(b + b_rp), b + b_rp + b_ci, R->n, R->nnz,
                        nullptr, nullptr, ts, &c) == cudaSuccess)
      best = c;
    cudaStreamSynchronize(ts);
    dev_free_on(b, ts);
  }
  cudaStreamDestroy(ts);
  return best;
}

// Offsets of a request's arrays in its staging block: row pointers, columns,
// values, lane sources and lengths, slices, lane outputs, cut rows.
struct StageLayout {
  size_t rp, ci, val, src, len, sl, out, lr, total;
};
StageLayout stage_offsets(const Request& R, size_t lanes, size_t slices, size_t lrows) {
  StageLayout L{};
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off = al256(off + std::max<size_t>(b, 1));
    return o;
  };
  L.rp = take((size_t)(R.n + 1) * 8);
  L.ci = take((size_t)R.nnz * 4);
  L.val = take(R.val_bytes);
  L.src = take(lanes * 8);
  L.len = take(lanes * 4);
  L.sl = take(slices * sizeof(SellSlice));
  L.out = take(lanes * 4);
  L.lr = take(lrows * sizeof(LongRow));
  L.total = off;
  return L;
}
// the offsets of R's built layout
StageLayout stage_layout(const Request& R) {
  return stage_offsets(R, R.ls_lanes, R.ls_slices, R.ls_lrows);
}
// a block that holds R's arrays under any candidate layout: a row of length
// L > 0 gives at most L / vmax + 1 pieces, a window's pieces fill their
// slices but the last, cut rows number at most nnz / vmax
StageLayout stage_bound(const Request& R) {
  int vmin = TUNE_VMAX[0], wmin = TUNE_WINDOW[0];
  for (int c = 1; c < TUNE_N; ++c) {
    vmin = std::min(vmin, TUNE_VMAX[c]);
    wmin = std::min(wmin, TUNE_WINDOW[c]);
  }
  const size_t pieces = (size_t)R.n + (size_t)R.nnz / (size_t)vmin;
  const size_t nwin = (size_t)((R.n + wmin - 1) / wmin);
  const size_t slices = pieces / SELL_C + nwin + 1;
  return stage_offsets(R, slices * SELL_C, slices, (size_t)R.nnz / (size_t)vmin + 1);
}

// Take R's block of the staging area, sized by stage_bound, in submission
// order (waiting while the area is full: admissions free it in that order,
// so the head of the queue always progresses).  Called when an analysis
// thread picks R up, so a thread waits only for the blocks of earlier
// requests, not for their layouts.  A request larger than the whole area is
// not staged (its copies run at admission).
void stage_reserve(te_server* S, Request* R) {
  const size_t bytes = stage_bound(*R).total;
  const double w0 = now_s();
  {
    std::unique_lock<std::mutex> lk(S->stage_mu);
    S->stage_cv.wait(lk, [&] { return S->stopping || S->stage_turn == R->seq; });
    if (S->stopping) return;
    if (bytes <= S->stage.size) {
      size_t off = 0;
      S->stage_cv.wait(lk, [&] { return S->stopping || S->stage.alloc(bytes, &off); });
      if (!S->stopping) {
        R->stage_off = off;
        R->stage_bytes = bytes;
      }
    }
    S->stage_turn += 1;
  }
  S->stage_cv.notify_all();
  S->a_wait_ns += (int64_t)((now_s() - w0) * 1e9);
}

// Copy R's CSR and built layout into its staging block: gathered by the CPU
// into the thread's pinned bounce buffer, then one DMA on the thread's stream
// (array by array from pageable memory when the buffer cannot hold them).
void stage_fill(te_server* S, Request* R, cudaStream_t ts, Bounce* B) {
  if (!R->stage_bytes) return;
  const StageLayout L = stage_layout(*R);
  const SellHost& H = R->layout;
  char* G = S->stage.base + R->stage_off;
  const double c0 = now_s();
  const bool bounced = L.total <= BOUNCE_MAX && B->reserve(L.total);
  if (bounced) {
    auto put = [&](size_t o, const void* src, size_t b) {
      if (b) std::memcpy(B->p + o, src, b);
    };
    put(L.rp, R->rp, (size_t)(R->n + 1) * 8);
    put(L.ci, R->ci, (size_t)R->nnz * 4);
    put(L.val, R->vals, R->val_bytes);
    put(L.src, H.vsrc.data(), H.vsrc.size() * 8);
    put(L.len, H.vlen.data(), H.vlen.size() * 4);
    put(L.sl, H.slices.data(), H.slices.size() * sizeof(SellSlice));
    put(L.out, H.vout.data(), H.vout.size() * 4);
    put(L.lr, H.lrows.data(), H.lrows.size() * sizeof(LongRow));
  }
  const double c1 = now_s();
  S->a_gather_ns += (int64_t)((c1 - c0) * 1e9);
  cudaError_t e = cudaSuccess;
  if (bounced) {
    e = cudaMemcpyAsync(G, B->p, L.total, cudaMemcpyHostToDevice, ts);
  } else {
    auto h2d = [&](size_t o, const void* src, size_t b) {
      if (e == cudaSuccess && b) e = cudaMemcpyAsync(G + o, src, b, cudaMemcpyHostToDevice, ts);
    };
    h2d(L.rp, R->rp, (size_t)(R->n + 1) * 8);
    h2d(L.ci, R->ci, (size_t)R->nnz * 4);
    h2d(L.val, R->vals, R->val_bytes);
    h2d(L.src, H.vsrc.data(), H.vsrc.size() * 8);
    h2d(L.len, H.vlen.data(), H.vlen.size() * 4);
    h2d(L.sl, H.slices.data(), H.slices.size() * sizeof(SellSlice));
    h2d(L.out, H.vout.data(), H.vout.size() * 4);
    h2d(L.lr, H.lrows.data(), H.lrows.size() * sizeof(LongRow));
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
  S->a_stage_ns += (int64_t)((now_s() - c1) * 1e9);
  if (e != cudaSuccess) {  // fall back to copies at admission
    (void)cudaGetLastError();
    std::lock_guard<std::mutex> lk(S->stage_mu);
    S->stage.release(R->stage_off, R->stage_bytes);
    R->stage_bytes = 0;
  }
}

// The request's CSR staged, then its SpMV layout built by the device layout
// kernels straight into its staging block (the same arrangement as
// make_sell's, element for element): the analysis thread only issues the
// copies and the kernels.  False (nothing recorded) when the request is not
// staged, the sizes are beyond the device build, or a call fails; the
// thread then builds the layout on the host.
bool analyse_on_device(te_server* S, Request* R, cudaStream_t ts, Bounce* B, int window,
                       int vmax) {
  if (!R->stage_bytes || !dev_layout_fits(R->n, window, vmax)) return false;
  const StageLayout L0 = stage_offsets(*R, 0, 0, 0);  // the CSR's offsets
  const size_t csr_bytes = L0.val + R->val_bytes;
  char* G = S->stage.base + R->stage_off;
  const double c0 = now_s();
  cudaError_t e = cudaSuccess;
  if (csr_bytes <= BOUNCE_MAX && B->reserve(csr_bytes)) {
    std::memcpy(B->p + L0.rp, R->rp, (size_t)(R->n + 1) * 8);
    if (R->nnz) std::memcpy(B->p + L0.ci, R->ci, (size_t)R->nnz * 4);
    if (R->val_bytes) std::memcpy(B->p + L0.val, R->vals, R->val_bytes);
    S->a_gather_ns += (int64_t)((now_s() - c0) * 1e9);
    e = cudaMemcpyAsync(G, B->p, csr_bytes, cudaMemcpyHostToDevice, ts);
  } else {
    e = cudaMemcpyAsync(G + L0.rp, R->rp, (size_t)(R->n + 1) * 8, cudaMemcpyHostToDevice, ts);
    if (e == cudaSuccess && R->nnz)
      e = cudaMemcpyAsync(G + L0.ci, R->ci, (size_t)R->nnz * 4, cudaMemcpyHostToDevice, ts);
    if (e == cudaSuccess && R->val_bytes)
      e = cudaMemcpyAsync(G + L0.val, R->vals, R->val_bytes, cudaMemcpyHostToDevice, ts);
  }
  const double c1 = now_s();
  DevLayout DL;
  std::string err;
  int64_t tot[4] = {0, 0, 0, 0};
  char* tmp = nullptr;
  int nbig = 0;
  bool ok = false;
  if (e == cudaSuccess)
    e = DL.count(reinterpret_cast<const int64_t*>(G + L0.rp), R->n, R->nnz, window, vmax, false,
                 ts, err);
  if (e == cudaSuccess) e = DL.windows(ts, tot);
  StageLayout L{};
  if (e == cudaSuccess) {
    L = stage_offsets(*R, (size_t)tot[0] * SELL_C, (size_t)tot[0], (size_t)tot[3]);
    ok = L.total <= R->stage_bytes;
  }
  if (ok) e = dev_alloc(&tmp, (size_t)std::max<int64_t>(tot[3], 1) * sizeof(LongRow));
  if (ok && e == cudaSuccess)
    e = DL.emit(reinterpret_cast<SellSlice*>(G + L.sl), reinterpret_cast<int32_t*>(G + L.out),
                reinterpret_cast<int64_t*>(G + L.src), reinterpret_cast<int32_t*>(G + L.len),
                nullptr, reinterpret_cast<LongRow*>(G + L.lr), reinterpret_cast<LongRow*>(tmp),
                ts, &nbig);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
  // the scratch goes back to the pool in stream order (no device-wide wait)
  if (tmp) dev_free_on(tmp, ts);
  if (DL.scratch) {
    dev_free_on(DL.scratch, ts);
    DL.scratch = nullptr;
  }
  S->a_layout_ns += (int64_t)((now_s() - c1) * 1e9);
  if (e != cudaSuccess || !ok) {
    (void)cudaGetLastError();
    return false;
  }
  R->ls_slices = (size_t)tot[0];
  R->ls_lanes = (size_t)tot[0] * SELL_C;
  R->ls_lrows = (size_t)tot[3];
  R->ls_entries = tot[1];
  R->ls_pieces = tot[2];
  return true;
}

// An analysis thread's work: the request's layout, with its class's tuned
// candidate when the server tunes (the class's first request is tuned here;
// others of the class wait for it), then its staging
void analyse_request(te_server* S, Request* R, cudaStream_t ts, Bounce* B) {
  stage_reserve(S, R);
  int cand = 0;
  if (S->autotune) {
    const int key = request_class(R);
    std::unique_lock<std::mutex> lk(S->tune_mu);
    for (;;) {
      auto it = S->tuned.find(key);
      if (it != S->tuned.end()) {
        cand = it->second;
        break;
      }
      if (!S->tuning.count(key)) {
        S->tuning.insert(key);
        lk.unlock();
        const int c = tune_request(R);
        lk.lock();
        S->tuning.erase(key);
        if (c >= 0) S->tuned[key] = c;  // an untunable request leaves the class open
        S->tune_cv.notify_all();
        cand = c >= 0 ? c : 0;
        break;
      }
      S->tune_cv.wait(lk);
    }
  }
  R->cand = cand;
  if (analyse_on_device(S, R, ts, B, TUNE_WINDOW[cand], TUNE_VMAX[cand])) {
    S->a_count += 1;
    return;
  }
  std::string perr;
  const double t0 = now_s();
  make_sell(R->rp, R->n, R->nnz, R->layout, perr, TUNE_WINDOW[cand], TUNE_VMAX[cand]);
  {
    const SellHost& H = R->layout;
    R->ls_slices = H.slices.size();
    R->ls_lanes = H.vout.size();
    R->ls_lrows = H.lrows.size();
    R->ls_entries = H.entries;
    R->ls_pieces = H.pieces;
  }
  S->a_layout_ns += (int64_t)((now_s() - t0) * 1e9);
  R->cand = cand;
  stage_fill(S, R, ts, B);
  S->a_count += 1;
}

// the batched step: SpMV (+ cut rows), three passes, three restart passes
cudaError_t enqueue_step(te_server* S, cudaStream_t s) {
  cudaError_t e = launch_batch_spmv(S->table_d, S->spmv_blocks, S->fin_blocks, s);
  for (int restart = 0; restart < 2 && e == cudaSuccess; ++restart) {
    if (e == cudaSuccess) e = launch_batch_pass(MODE_DOT, S->table_d, restart, S->Lpass, s);
    if (e == cudaSuccess) e = launch_batch_pass(MODE_AXPY_DOT, S->table_d, restart, S->Lpass, s);
    if (e == cudaSuccess)
      e = launch_batch_pass(MODE_AXPY_STORE, S->table_d, restart, S->Lpass, s);
  }
  return e;
}

// device work memory of a request: the SELL copy, the solver vectors and
// state; `tmp`: what only the admission needs; `res`: the Ritz vectors
struct AdmitLayout {
  size_t slices, vout, cols, vals, lrows, vpart, V, ytil, w, partials, st, flag, total;
  size_t t_rp, t_ci, t_val, t_src, t_len, t_q, t_total;
};

AdmitLayout admit_layout(const Request& R, const SellHost& H) {
  const bool staged = R.stage_bytes > 0;  // the staging area holds the CSR and lane map
  AdmitLayout L{};
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off = al256(off + std::max<size_t>(b, 1));
    return o;
  };
  const size_t velt = R.vk == TE_BF16 ? 2 : 4;
  L.slices = take(R.ls_slices * sizeof(SellSlice));
  L.vout = take(R.ls_lanes * sizeof(int32_t));
  L.cols = take((size_t)R.ls_entries * 4);
  L.vals = take((size_t)R.ls_entries * velt);
  L.lrows = take(R.ls_lrows * sizeof(LongRow));
  L.vpart = take((size_t)R.ls_pieces * 8);
  L.V = take((size_t)R.n_pad * (R.m + 1) * 4);
  L.ytil = take((size_t)R.n_pad * 8);
  L.w = take((size_t)R.n_pad * 8);
  L.partials = take((size_t)R.ncta * PSTRIDE * 8);
  L.st = take(sizeof(LzState));
  L.flag = take(16);
  L.total = off;
  off = 0;
  L.t_rp = take(staged ? 0 : (size_t)(R.n + 1) * 8);
  L.t_ci = take(staged ? 0 : (size_t)R.nnz * 4);
  L.t_val = take(staged ? 0 : (size_t)R.nnz * (R.in_type == TE_F64 ? 8 : 4));
  L.t_src = take(staged ? 0 : R.ls_lanes * 8);
  L.t_len = take(staged ? 0 : R.ls_lanes * 4);
  L.t_q = take(R.vk == TE_BF16 ? (size_t)R.nnz * 2 : 0);
  L.t_total = off;
  return L;
}

// Try to admit R into slot k.  Returns 1 on success, 0 when the pool has no
// room now, -1 on a CUDA error (status set).
int admit(te_server* S, Request* R, int k, te_status* err) {
  const SellHost& H = R->layout;  // built by an analysis thread
  const AdmitLayout L = admit_layout(*R, H);
  size_t work = 0, res = 0, tmp = 0;
  if (!S->pool.alloc(L.total, &work)) return 0;
  if (!S->pool.alloc((size_t)R->n * R->K * 8, &res)) {
    S->pool.release(work, L.total);
    return 0;
  }
  if (!S->pool.alloc(L.t_total, &tmp)) {
    S->pool.release(work, L.total);
    S->pool.release(res, (size_t)R->n * R->K * 8);
    return 0;
  }
  R->work_off = work;
  R->work_bytes = L.total;
  R->res_off = res;
  R->res_bytes = (size_t)R->n * R->K * 8;
  S->deferred.push_back({tmp, L.t_total});
  char* W = S->pool.base + work;
  char* T = S->pool.base + tmp;
  cudaStream_t s = S->as;  // beside the engine step
  cudaError_t e = cudaMemsetAsync(W, 0, L.total, s);
  // the CSR and layout: in the staging area (copied by the analysis thread)
  // or copied from the host now
  const bool staged = R->stage_bytes > 0;
  const StageLayout G = stage_layout(*R);
  const char* GB = S->stage.base + R->stage_off;
  auto h2d = [&](void* dst, const void* src, size_t b) {
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s);
  };
  if (!staged) {
    h2d(T + L.t_rp, R->rp, (size_t)(R->n + 1) * 8);
    h2d(T + L.t_ci, R->ci, (size_t)R->nnz * 4);
    h2d(T + L.t_val, R->vals, R->val_bytes);
    h2d(T + L.t_src, H.vsrc.data(), H.vsrc.size() * 8);
    h2d(T + L.t_len, H.vlen.data(), H.vlen.size() * 4);
  }
  const int64_t* drp = reinterpret_cast<const int64_t*>(staged ? GB + G.rp : T + L.t_rp);
  const int32_t* dci = reinterpret_cast<const int32_t*>(staged ? GB + G.ci : T + L.t_ci);
  const void* dval = staged ? (const void*)(GB + G.val) : (const void*)(T + L.t_val);
  const int64_t* dsrc = reinterpret_cast<const int64_t*>(staged ? GB + G.src : T + L.t_src);
  const int32_t* dlen = reinterpret_cast<const int32_t*>(staged ? GB + G.len : T + L.t_len);
  // column indices are checked here, before the solve's first SpMV (the
  // request joins the batch only after the next step has read the flag)
  int* flag = reinterpret_cast<int*>(W + L.flag);
  if (e == cudaSuccess) e = launch_validate_cols(dci, R->nnz, R->n, flag, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&S->res_h[k].bad_cols, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (staged) {
    auto d2d = [&](void* dst, const void* src, size_t b) {
      if (e == cudaSuccess && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, s);
    };
    d2d(W + L.slices, GB + G.sl, R->ls_slices * sizeof(SellSlice));
    d2d(W + L.vout, GB + G.out, R->ls_lanes * 4);
    d2d(W + L.lrows, GB + G.lr, R->ls_lrows * sizeof(LongRow));
  } else {
    h2d(W + L.slices, H.slices.data(), H.slices.size() * sizeof(SellSlice));
    h2d(W + L.vout, H.vout.data(), H.vout.size() * 4);
    h2d(W + L.lrows, H.lrows.data(), H.lrows.size() * sizeof(LongRow));
  }
  const void* vin = dval;
  int in_type = R->in_type;
  if (e == cudaSuccess && R->vk == TE_BF16) {
    e = launch_quantize(TE_BF16, drp, static_cast<const double*>(dval), R->n, R->nnz, T + L.t_q,
                        nullptr, s);
    vin = T + L.t_q;
    in_type = TE_BF16;
  }
  if (e == cudaSuccess)
    e = launch_sell_fill_cols(dci, reinterpret_cast<const SellSlice*>(W + L.slices), dsrc, dlen,
                              (int)R->ls_slices, reinterpret_cast<int32_t*>(W + L.cols),
                              nullptr, nullptr, s);
  if (e == cudaSuccess)
    e = launch_sell_fill_vals(in_type, R->vk, vin, reinterpret_cast<const SellSlice*>(W + L.slices),
                              dsrc, dlen, (int)R->ls_slices, W + L.vals, nullptr, nullptr,
                              nullptr, nullptr, s);
  LzState* st = reinterpret_cast<LzState*>(W + L.st);
  double* U = reinterpret_cast<double*>(S->pool.base + res);
  if (e == cudaSuccess) e = launch_solve_begin(st, nullptr, U, nullptr, nullptr, s);
  // the start vector: stream 0 of the seed, normalised (the init pass)
  BatchSlot& B = R->desc;
  B.slices = reinterpret_cast<const SellSlice*>(W + L.slices);
  B.vout = reinterpret_cast<const int32_t*>(W + L.vout);
  B.cols = reinterpret_cast<const int32_t*>(W + L.cols);
  B.vals = W + L.vals;
  B.lrows = reinterpret_cast<const LongRow*>(W + L.lrows);
  B.vpart = W + L.vpart;
  B.V = W + L.V;
  B.ytil = W + L.ytil;
  B.w = W + L.w;
  B.partials = W + L.partials;
  B.st = st;
  B.n = R->n;
  B.n_pad = R->n_pad;
  B.seed = R->seed;
  B.tol = breakdown_tolerance(PREC_FDF);
  B.vk = R->vk;
  B.nslices = (int)R->ls_slices;
  B.nlrows = (int)R->ls_lrows;
  B.m = R->m;
  B.K = R->K;
  B.step = 0;
  B.ncta = R->ncta;
  if (e == cudaSuccess) {
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.V = B.V;
    a.Vmut = B.V;
    a.ld = B.n_pad;
    a.tstride = TILE_R;  // column-major
    a.cstride = B.n_pad;
    a.n = B.n;
    a.m = B.m;
    a.K = B.K;
    a.seed = B.seed;
    a.tol = B.tol;
    a.st = st;
    a.partials = B.partials;
    a.nb = 0;
    a.col_out = 0;
    a.xsrc = X_V1;
    a.fin = FIN_STORE_INIT;
    PassLaunch Li = S->Lsto;
    Li.grid = R->ncta;
    e = launch_pass(PREC_FDF, MODE_AXPY_STORE, a, Li, s);
  }
  if (e != cudaSuccess) {
    *err = srv_cuda(e, "admission");
    return -1;
  }
  R->slot = k;
  R->state = REQ_ADMITTED;
  R->step = 0;
  // (the host arrangement is dropped once the admission kernels are done:
  // with host_direct they read it in place)
  return 1;
}

// A request's Ritz vectors to a caller's pinned buffer, stored by a few SMs
// through the buffer's device mapping (over NVLink-C2C): faster than a
// device-to-host copy-engine transfer, and few enough CTAs to leave the
// engine's kernels their SMs.
constexpr int POLL_COPY_CTAS = 16;
__global__ void __launch_bounds__(256) poll_copy_kernel(const double2* __restrict__ src,
                                                        double2* __restrict__ dst, int64_t n2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// the device address of pinned host memory, else NULL (pageable memory)
void* pinned_device_ptr(void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Jacobi, selection and Ritz vectors of a solve that completed its m steps,
// then its eigenvalues, residual estimates and status to the pinned slot area
cudaError_t enqueue_finish(te_server* S, Request* R, cudaStream_t fs) {
  const BatchSlot& B = R->desc;
  JacobiArgs j;
  memset(&j, 0, sizeof(j));
  j.alpha = B.st->alpha;
  j.beta = B.st->beta;
  j.s = B.st->s;
  j.m = B.m;
  j.K = B.K;
  j.which = TE_WHICH_LARGEST_MAGNITUDE;
  j.theta_out = B.st->theta_sel;
  j.C_out = B.st->C;
  j.resid_out = B.st->resid_est;
  j.st = B.st;
  cudaError_t e = launch_jacobi(j, fs);
  if (e == cudaSuccess) {
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.V = B.V;
    a.Vmut = B.V;
    a.ld = B.n_pad;
    a.tstride = TILE_R;  // column-major
    a.cstride = B.n_pad;
    a.n = B.n;
    a.m = B.m;
    a.K = B.K;
    a.st = B.st;
    a.partials = B.partials;
    a.nb = B.m;
    a.fin = FIN_NONE;
    PassLaunch Lr = S->Lritz;
    Lr.grid = R->ncta;
    e = launch_pass(PREC_FDF, MODE_RITZ, a, Lr, fs);
  }
  SlotResult* out = S->res_h + R->slot;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out->theta, B.st->theta_sel, sizeof(double) * B.K, cudaMemcpyDeviceToHost,
                        fs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out->resid, B.st->resid_est, sizeof(double) * B.K,
                        cudaMemcpyDeviceToHost, fs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out->hdr, &B.st->restart_flag, sizeof(out->hdr), cudaMemcpyDeviceToHost,
                        fs);
  return e;
}

te_status check_request(const te_csr* A, int32_t K, int32_t m, te_precision p, int max_m) {
  if (!A) return srv_fail(TE_ERR_INVALID_ARG, "A is NULL");
  if (A->where != TE_HOST) return srv_fail(TE_ERR_INVALID_ARG, "the server takes host matrices");
  if (A->n < 1 || A->n >= (int64_t)1 << 31 || A->nnz < 0)
    return srv_fail(TE_ERR_INVALID_ARG, "n or nnz out of range");
  if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->values)))
    return srv_fail(TE_ERR_INVALID_ARG, "CSR arrays must not be NULL");
  if (A->row_scale) return srv_fail(TE_ERR_UNSUPPORTED, "row_scale is reserved (must be NULL)");
  if (!(p.arithmetic == TE_F64 && p.vectors == TE_F32 &&
        (p.values == TE_F32 || p.values == TE_BF16)))
    return srv_fail(TE_ERR_UNSUPPORTED, "the server runs FDF and BDF");
  if (p.values == TE_BF16 && A->values_f64 != 1)
    return srv_fail(TE_ERR_INVALID_ARG, "bfloat16 storage is built from binary64 values");
  if (K < 1 || m < K || (int64_t)m > A->n)
    return srv_fail(TE_ERR_INVALID_ARG, "need 1 <= K <= krylov_steps <= n");
  if (m > max_m) return srv_fail(TE_ERR_UNSUPPORTED, "krylov_steps above the server's maximum");
  return TE_OK;
}

}  // namespace

extern "C" {

te_status te_server_create(const te_server_options* o, te_server** out) {
  if (!o || !out) return srv_fail(TE_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (o->max_slots < 1 || o->max_slots > SRV_MAX_SLOTS)
    return srv_fail(TE_ERR_INVALID_ARG, "max_slots must be in [1, 64]");
  if (o->max_krylov_steps < 1 || o->max_krylov_steps > MAX_M)
    return srv_fail(TE_ERR_INVALID_ARG, "max_krylov_steps must be in [1, 64]");
  if (o->device_budget_bytes < ((size_t)1 << 20))
    return srv_fail(TE_ERR_INVALID_ARG, "device_budget_bytes must be at least 1 MiB");
  if (o->autotune != 0 && o->autotune != 1)
    return srv_fail(TE_ERR_INVALID_ARG, "autotune must be 0 or 1");
  te_server* S = new te_server();
  struct Guard {
    te_server*& p;
    bool keep = false;
    ~Guard() {
      if (!keep) te_server_destroy(p);
    }
  } guard{S};
  S->max_slots = o->max_slots;
  S->max_m = o->max_krylov_steps;
  S->autotune = o->autotune != 0;
  S->use_graph = o->use_graph != 0;
  S->slots.assign(S->max_slots, nullptr);
  int dev = 0;
  SRV_CK(cudaGetDevice(&dev), "cudaGetDevice");
  S->dev = dev;
  SRV_CK(cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
  {
    size_t sb = o->device_budget_bytes / 8;
    sb = std::max<size_t>(sb, (size_t)64 << 20);
    sb = std::min<size_t>(sb, (size_t)2 << 30);
    SRV_CK(S->stage.init(sb), "allocate the staging area");
  }

  SRV_CK(cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking), "create stream");
  SRV_CK(cudaStreamCreateWithFlags(&S->ps, cudaStreamNonBlocking), "create stream");
  SRV_CK(cudaStreamCreateWithFlags(&S->as, cudaStreamNonBlocking), "create stream");
  for (cudaStream_t& f : S->fs)
    SRV_CK(cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking), "create stream");
  SRV_CK(batch_spmv_grids(S->num_sms, &S->spmv_blocks, &S->fin_blocks), "size the SpMV grids");
  SRV_CK(cudaEventCreateWithFlags(&S->ev_step, cudaEventDisableTiming), "create event");
  SRV_CK(cudaEventCreateWithFlags(&S->ev_admit, cudaEventDisableTiming), "create event");
  SRV_CK(cudaEventCreateWithFlags(&S->ev, cudaEventDisableTiming), "create event");
  SRV_CK(S->pool.init(o->device_budget_bytes), "allocate the device pool");
  SRV_CK(cudaMallocHost(&S->table_h, sizeof(BatchTable)), "allocate the step table");
  SRV_CK(cudaMalloc(&S->table_d, sizeof(BatchTable)), "allocate the step table");
  SRV_CK(cudaMallocHost(&S->res_h, sizeof(SlotResult) * SRV_MAX_SLOTS), "allocate results");
  memset(S->table_h, 0, sizeof(BatchTable));
  SRV_CK(cudaMemcpy(S->table_d, S->table_h, sizeof(BatchTable), cudaMemcpyHostToDevice),
         "clear the step table");
  SRV_CK(jacobi_prepare(), "kernel set-up");
  SRV_CK(pass_config(PREC_FDF, MODE_AXPY_DOT, S->max_m, 1, S->num_sms, S->Lpass),
         "configure passes");
  SRV_CK(pass_config(PREC_FDF, MODE_AXPY_STORE, S->max_m, 1, S->num_sms, S->Lsto),
         "configure passes");
  SRV_CK(pass_config(PREC_FDF, MODE_RITZ, S->max_m, S->max_m, S->num_sms, S->Lritz),
         "configure passes");
  SRV_CK(pass_config(PREC_FDF, MODE_DOT, S->max_m, 1, S->num_sms, S->Lpass), "configure passes");
  SRV_CK(batch_pass_prepare(S->Lpass), "configure batched passes");
  {
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt > 2 ? nt / 2 : 1;
    if (nt > 8) nt = 8;
    S->analysis.start(nt, dev, [S](Request* R, cudaStream_t ts, Bounce* B) {
      analyse_request(S, R, ts, B);
    });
  }
  if (S->use_graph) {
    cudaGraph_t g = nullptr;
    SRV_CK(cudaStreamBeginCapture(S->s, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_step(S, S->s);
    cudaError_t e2 = cudaStreamEndCapture(S->s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return srv_cuda(e != cudaSuccess ? e : e2, "capture the engine step");
    }
    e = cudaGraphInstantiate(&S->gexec, g, 0);
    cudaGraphDestroy(g);
    SRV_CK(e, "instantiate the engine step");
  }
  guard.keep = true;
  *out = S;
  return TE_OK;
}

void te_server_destroy(te_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->stage_mu);
    S->stopping = true;
  }
  S->stage_cv.notify_all();
  S->analysis.stop();  // no thread touches a request after this
  if (S->s) cudaStreamSynchronize(S->s);
  if (S->as) cudaStreamSynchronize(S->as);
  for (cudaStream_t f : S->fs)
    if (f) cudaStreamSynchronize(f);
  for (auto& kv : S->reqs) delete kv.second;
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  if (S->ev) cudaEventDestroy(S->ev);
  if (S->table_h) cudaFreeHost(S->table_h);
  if (S->table_d) cudaFree(S->table_d);
  if (S->res_h) cudaFreeHost(S->res_h);
  if (S->s) cudaStreamDestroy(S->s);
  if (S->as) cudaStreamDestroy(S->as);
  for (cudaStream_t f : S->fs)
    if (f) cudaStreamDestroy(f);
  if (S->ev_step) cudaEventDestroy(S->ev_step);
  for (auto& b : S->batches) cudaEventDestroy(b.ev);
  for (cudaEvent_t e : S->ev_free) cudaEventDestroy(e);
  if (S->ev_admit) cudaEventDestroy(S->ev_admit);
  if (S->ps) cudaStreamDestroy(S->ps);
  delete S;
}

te_status te_server_submit(te_server* S, const te_csr* A, int32_t K, int32_t m, te_precision p,
                           uint64_t seed, int64_t* ticket) {
  if (!S || !ticket) return srv_fail(TE_ERR_INVALID_ARG, "NULL argument");
  const double t0 = now_s();
  struct Acc {
    double t0;
    double& acc;
    ~Acc() { acc += now_s() - t0; }
  } acc{t0, S->t_submit};
  te_status r = check_request(A, K, m, p, S->max_m);
  if (r != TE_OK) return r;
  // row pointers are checked now (the layout is built from them); column
  // indices on the device at admission
  const int64_t* rp = A->row_ptr;
  if (rp[0] != 0 || rp[A->n] != A->nnz) return srv_fail(TE_ERR_INVALID_ARG, "malformed row_ptr");
  for (int64_t i = 0; i < A->n; ++i)
    if (rp[i + 1] < rp[i]) return srv_fail(TE_ERR_INVALID_ARG, "row_ptr must be non-decreasing");
  Request* R = new Request();
  R->ticket = S->next_ticket++;
  R->n = A->n;
  R->nnz = A->nnz;
  R->n_pad = pad_rows(A->n);
  R->K = K;
  R->m = m;
  R->seed = seed;
  R->vk = p.values;
  R->in_type = A->values_f64 ? TE_F64 : TE_F32;
  R->ncta = ctas_for(R->n_pad);
  R->rp = rp;
  R->ci = A->col_idx;
  R->vals = A->values;
  R->val_bytes = (size_t)A->nnz * (R->in_type == TE_F64 ? 8 : 4);
  R->seq = S->next_seq++;
  S->reqs[R->ticket] = R;
  S->pending.push_back(R);
  S->analysis.post(R);
  *ticket = R->ticket;
  return TE_OK;
}

te_status te_server_step(te_server* S, int32_t* live_out, int32_t* pending_out) {
  if (!S) return srv_fail(TE_ERR_INVALID_ARG, "server is NULL");
  double t0 = now_s();
  // 1. the previous step has finished: retire the solves that ended in it,
  //    and let the requests admitted in it join the batch (or fail them)
  if (S->inflight) {
    SRV_CK(cudaEventSynchronize(S->ev), "engine step");
    S->inflight = false;
  }
  // finished Jacobi / Ritz batches, oldest first; block on the oldest only
  // when no solve is stepping (so that a client waiting for results moves on)
  {
    bool stepping = false, free_slot = false;
    for (Request* R : S->slots) {
      stepping |= R && (R->state == REQ_RUNNING || R->state == REQ_ADMITTED);
      free_slot |= R == nullptr;
    }
    bool retired = false;
    for (auto it = S->batches.begin(); it != S->batches.end();) {
      te_server::FinishBatch& b = *it;
      cudaError_t q = cudaEventQuery(b.ev);
      if (q == cudaErrorNotReady) {
        // the batches run on several streams: a later one may be done first
        if (stepping || retired || (free_slot && !S->pending.empty()) ||
            it != S->batches.begin()) {
          ++it;
          continue;
        }
        q = cudaEventSynchronize(b.ev);
      }
      SRV_CK(q, "finish solves");
      retired = true;
      for (int k : b.slots) {
        Request* R = S->slots[k];
        const SlotResult& o = S->res_h[k];
        R->theta.assign(o.theta, o.theta + R->K);
        R->resid.assign(o.resid, o.resid + R->K);
        R->status = o.hdr[2];
        R->state = REQ_FINISHED;
        S->completed.push_back(R->ticket);
        S->pool.release(R->work_off, R->work_bytes);
        S->slots[k] = nullptr;
        R->slot = -1;
      }
      S->ev_free.push_back(b.ev);
      it = S->batches.erase(it);
    }
  }
  // the admissions of the previous call ran on their own stream
  if (S->admit_pending) {
    SRV_CK(cudaEventSynchronize(S->ev_admit), "admission");
    S->admit_pending = false;
    for (auto& d : S->deferred) S->pool.release(d.first, d.second);
    S->deferred.clear();
    for (int k = 0; k < S->max_slots; ++k) {
      Request* R = S->slots[k];
      if (!R || R->state != REQ_ADMITTED) continue;
      R->layout = SellHost();  // its admission kernels are done
      if (R->stage_bytes) {
        {
          std::lock_guard<std::mutex> lk(S->stage_mu);
          S->stage.release(R->stage_off, R->stage_bytes);
          R->stage_bytes = 0;
        }
        S->stage_cv.notify_all();
      }
      if (S->res_h[k].bad_cols) {
        R->status = TE_ERR_INVALID_ARG;
        R->state = REQ_FINISHED;
        S->completed.push_back(R->ticket);
        S->pool.release(R->work_off, R->work_bytes);
        S->pool.release(R->res_off, R->res_bytes);
        R->res_bytes = 0;
        S->slots[k] = nullptr;
        R->slot = -1;
      } else {
        R->state = REQ_RUNNING;
      }
    }
  }
  double t1 = now_s();
  S->t_wait += t1 - t0;
  // 2. one Lanczos step of every resident solve
  BatchTable* T = S->table_h;
  int ns = 0;
  T->slice_off[0] = 0;
  T->lrow_off[0] = 0;
  T->item_off[0] = 0;
  for (int k = 0; k < S->max_slots; ++k) {
    Request* R = S->slots[k];
    if (!R || R->state != REQ_RUNNING) continue;
    R->desc.step = R->step;
    T->slot[ns] = R->desc;
    T->slice_off[ns + 1] = T->slice_off[ns] + R->desc.nslices;
    T->lrow_off[ns + 1] = T->lrow_off[ns] + R->desc.nlrows;
    T->item_off[ns + 1] = T->item_off[ns] + R->desc.ncta;
    ++ns;
  }
  T->nslots = ns;
  if (ns > 0) {
    S->engine_steps += 1;
    S->resident_steps += ns;
    SRV_CK(cudaMemcpyAsync(S->table_d, T, sizeof(BatchTable), cudaMemcpyHostToDevice, S->s),
           "upload the step table");
    if (S->gexec) SRV_CK(cudaGraphLaunch(S->gexec, S->s), "launch the engine step");
    else SRV_CK(enqueue_step(S, S->s), "engine step");
    // solves that completed their m steps: Jacobi and Ritz vectors on the
    // finishing stream, after this step
    te_server::FinishBatch batch[te_server::SRV_FIN_STREAMS];
    bool recorded = false;
    for (int k = 0; k < S->max_slots; ++k) {
      Request* R = S->slots[k];
      if (!R || R->state != REQ_RUNNING) continue;
      R->step += 1;
      if (R->step == R->m) {
        if (!recorded) {
          SRV_CK(cudaEventRecord(S->ev_step, S->s), "record");
          recorded = true;
        }
        const int f = S->fs_next;
        S->fs_next = (f + 1) % te_server::SRV_FIN_STREAMS;
        if (batch[f].slots.empty())
          SRV_CK(cudaStreamWaitEvent(S->fs[f], S->ev_step, 0), "wait");
        SRV_CK(enqueue_finish(S, R, S->fs[f]), "finish a solve");
        R->state = REQ_FINISHING;
        batch[f].slots.push_back(k);
      }
    }
    for (int f = 0; f < te_server::SRV_FIN_STREAMS; ++f) {
      if (batch[f].slots.empty()) continue;
      if (S->ev_free.empty()) {
        cudaEvent_t e = nullptr;
        SRV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create event");
        S->ev_free.push_back(e);
      }
      batch[f].ev = S->ev_free.back();
      S->ev_free.pop_back();
      SRV_CK(cudaEventRecord(batch[f].ev, S->fs[f]), "record");
      S->batches.push_back(std::move(batch[f]));
    }
  }
  double t2 = now_s();
  S->t_launch += t2 - t1;
  // 3. admit in submission order while a slot and pool memory are free; the
  //    host work overlaps the step just launched, the uploads follow it
  int live = 0;
  bool admitted = false;
  for (Request* R : S->slots) live += R != nullptr;
  while (!S->pending.empty() && live < S->max_slots) {
    Request* R = S->pending.front();
    if (!R->analysed.load(std::memory_order_acquire)) {
      // in submission order: wait for the head's layout only when nothing
      // else would run (otherwise it is admitted at a later step)
      if (live > 0) break;
      S->analysis.wait(R);
    }
    int k = 0;
    while (S->slots[k]) ++k;
    te_status err = TE_OK;
    const int a = admit(S, R, k, &err);
    if (a < 0) return err;
    if (a == 0) {
      if (live == 0 && S->pool.used == 0) {
        // nothing resident and the pool is empty: this request can never fit
        R->status = TE_ERR_OUT_OF_MEMORY;
        R->state = REQ_FINISHED;
        S->completed.push_back(R->ticket);
        if (R->stage_bytes) {
          {
            std::lock_guard<std::mutex> lk(S->stage_mu);
            S->stage.release(R->stage_off, R->stage_bytes);
            R->stage_bytes = 0;
          }
          S->stage_cv.notify_all();
        }
        S->pending.pop_front();
        continue;
      }
      break;
    }
    S->pending.pop_front();
    S->slots[k] = R;
    ++live;
    admitted = true;
  }
  if (admitted) {
    SRV_CK(cudaEventRecord(S->ev_admit, S->as), "record");
    S->admit_pending = true;
  }
  S->t_admit += now_s() - t2;
  if (live_out) *live_out = live;
  if (pending_out) *pending_out = (int32_t)S->pending.size();
  if (live > 0) {
    SRV_CK(cudaEventRecord(S->ev, S->s), "record");
    S->inflight = true;
  }
  return TE_OK;
}

te_status te_server_timing(const te_server* S, double* wait_s, double* admit_s, double* launch_s,
                           double* submit_s, double* poll_copy_s, double* poll_free_s) {
  if (!S) return srv_fail(TE_ERR_INVALID_ARG, "server is NULL");
  if (wait_s) *wait_s = S->t_wait;
  if (admit_s) *admit_s = S->t_admit;
  if (launch_s) *launch_s = S->t_launch;
  if (submit_s) *submit_s = S->t_submit;
  if (poll_copy_s) *poll_copy_s = S->t_poll_copy;
  if (poll_free_s) *poll_free_s = S->t_poll_free;
  return TE_OK;
}

te_status te_server_analysis(const te_server* S, double* layout_s, double* gather_s,
                             double* copy_s, double* stage_wait_s, int64_t* analysed,
                             int64_t* engine_steps, int64_t* resident_steps) {
  if (!S) return srv_fail(TE_ERR_INVALID_ARG, "server is NULL");
  if (layout_s) *layout_s = 1e-9 * (double)S->a_layout_ns.load();
  if (gather_s) *gather_s = 1e-9 * (double)S->a_gather_ns.load();
  if (copy_s) *copy_s = 1e-9 * (double)S->a_stage_ns.load();
  if (stage_wait_s) *stage_wait_s = 1e-9 * (double)S->a_wait_ns.load();
  if (analysed) *analysed = S->a_count.load();
  if (engine_steps) *engine_steps = S->engine_steps;
  if (resident_steps) *resident_steps = S->resident_steps;
  return TE_OK;
}

te_status te_server_poll(te_server* S, int64_t ticket, int32_t* done, double* eigvals,
                         double* eigvecs, double* residuals) {
  if (!S || !done) return srv_fail(TE_ERR_INVALID_ARG, "NULL argument");
  *done = 0;
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return srv_fail(TE_ERR_INVALID_ARG, "unknown ticket");
  Request* R = it->second;
  if (R->state != REQ_FINISHED) return TE_OK;
  *done = 1;
  te_status st = (te_status)R->status;
  const double p0 = now_s();
  if (R->res_bytes) {
    if ((st == TE_OK || st == TE_ERR_BREAKDOWN) && eigvecs) {
      cudaError_t e = cudaSuccess;
      void* mapped = pinned_device_ptr(eigvecs);
      const char* src = S->pool.base + R->res_off;
      if (mapped && ((reinterpret_cast<uintptr_t>(mapped) | reinterpret_cast<uintptr_t>(src)) &
                     15) == 0 && R->res_bytes % 16 == 0) {
        poll_copy_kernel<<<POLL_COPY_CTAS, 256, 0, S->ps>>>(
            reinterpret_cast<const double2*>(src), static_cast<double2*>(mapped),
            (int64_t)(R->res_bytes / 16));
        e = cudaGetLastError();
      } else {
        e = cudaMemcpyAsync(eigvecs, src, R->res_bytes, cudaMemcpyDeviceToHost, S->ps);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(S->ps);
      if (e != cudaSuccess) return srv_cuda(e, "copy the Ritz vectors");
    }
    S->pool.release(R->res_off, R->res_bytes);
  }
  if (st == TE_OK || st == TE_ERR_BREAKDOWN) {
    if (eigvals) memcpy(eigvals, R->theta.data(), sizeof(double) * R->K);
    if (residuals) memcpy(residuals, R->resid.data(), sizeof(double) * R->K);
  }
  const double p1 = now_s();
  S->reqs.erase(it);
  delete R;
  S->t_poll_copy += p1 - p0;
  S->t_poll_free += now_s() - p1;
  if (st != TE_OK) return srv_fail(st, std::string("request failed: ") + te_status_string(st));
  return TE_OK;
}

te_status te_server_completed(te_server* S, int64_t* tickets, int32_t cap, int32_t* count) {
  if (!S || !count || cap < 0 || (cap > 0 && !tickets))
    return srv_fail(TE_ERR_INVALID_ARG, "bad arguments");
  int32_t c = 0;
  while (c < cap && !S->completed.empty()) {
    tickets[c++] = S->completed.front();
    S->completed.pop_front();
  }
  *count = c;
  return TE_OK;
}

te_status te_server_classes(te_server* S, int32_t* class_key, int32_t* window, int32_t* vmax,
                            int32_t cap, int32_t* count) {
  if (!S || !count || cap < 0) return srv_fail(TE_ERR_INVALID_ARG, "bad arguments");
  std::lock_guard<std::mutex> lk(S->tune_mu);
  int32_t c = 0;
  for (const auto& kv : S->tuned) {
    if (c < cap) {
      if (class_key) class_key[c] = kv.first;
      if (window) window[c] = TUNE_WINDOW[kv.second];
      if (vmax) vmax[c] = TUNE_VMAX[kv.second];
    }
    ++c;
  }
  *count = c;
  return TE_OK;
}

te_status te_server_stats(const te_server* S, int32_t* live, int32_t* pending, size_t* used,
                          size_t* peak) {
  if (!S) return srv_fail(TE_ERR_INVALID_ARG, "server is NULL");
  int n = 0;
  for (Request* R : S->slots) n += R != nullptr;
  if (live) *live = n;
  if (pending) *pending = (int32_t)S->pending.size();
  if (used) *used = S->pool.used;
  if (peak) *peak = S->pool.peak;
  return TE_OK;
}

}  // extern "C"
