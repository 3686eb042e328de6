// te_common.cuh - device-side building blocks shared by the sm_103a kernels of
// the Top-K Lanczos eigensolver: double-float ("dw") arithmetic on the FP32
// pipes, warp reductions, and thin inline-PTX wrappers for mbarriers and
// bulk (TMA) copies with bounded waits.
//
// Double-float arithmetic follows the error-free transformations of
// Dekker (1971) and Knuth (TwoSum), the compensated dot product "Dot2" of
// Ogita, Rump & Oishi (SIAM J. Sci. Comput. 26, 2005), and the double-word
// algorithms of Joldes, Muller & Popescu (ACM TOMS 44, 2017).  A dw value is
// the unevaluated sum hi + lo of two binary32 numbers (about 48 significant
// bits).  On this GPU the FP64 pipe runs at a small fraction of the FP32 one,
// so kernels that the paper asks to compute "in double precision" do their
// per-element work in dw and only cross-block sums in binary64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define TE_DEV __device__ __forceinline__

namespace te {

// ---------------------------------------------------------------------------
// error-free transformations (round-to-nearest intrinsics: no contraction)
// ---------------------------------------------------------------------------
TE_DEV void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// requires |a| >= |b| (or a == 0)
TE_DEV void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
TE_DEV void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

struct dw {
  float hi, lo;
};

TE_DEV dw dw_make(float h, float l) {
  dw r;
  fast_two_sum(h, l, r.hi, r.lo);
  return r;
}
TE_DEV dw dw_from_f2(float2 v) { return dw{v.x, v.y}; }
TE_DEV float2 dw_to_f2(dw v) { return make_float2(v.hi, v.lo); }

// exact split of a binary64 number into hi + lo (lo carries the next 24 bits)
TE_DEV dw dw_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return dw{h, l};
}
TE_DEV double dw_to_double(dw v) { return (double)v.hi + (double)v.lo; }

// The same value, hi + lo rounded to nearest binary64, built with integer
// operations (GB300 issues binary64 arithmetic and conversions at a small
// fraction of its binary32 rate).  Needs |lo| <= ulp(hi) / 2, as a two_sum
// leaves it.  hi's binary64 pattern is its sign, its exponent rebiased and
// its significand moved up 29 bits; lo is then added as a whole number of
// binary64 units in the last place of hi, 2^(e - 52), rounded to nearest
// even.  When hi is a power of two and lo lowers its magnitude, the result
// lies in the binade below, whose units are half as large.  Zeros,
// subnormals, infinities, NaNs and |hi| < 2^-74 take the binary64 path.
TE_DEV double dw_to_double_bits(dw v) {
  const uint32_t hb = __float_as_uint(v.hi);
  const uint32_t e8 = (hb >> 23) & 0xffu;
  if (e8 < 53u || e8 == 0xffu) return dw_to_double(v);
  const uint32_t mant = hb & 0x7fffffu;
  const bool opposite = ((__float_as_uint(v.lo) ^ hb) >> 31) != 0u;
  const uint32_t down = (mant == 0u && opposite) ? 1u : 0u;
  // 2^(52 - e + down) as a binary32, e = e8 - 127: exponent field 306 - e8 + down
  const float scale = __uint_as_float((306u - e8 + down) << 23);
  const int L = __float2int_rn(__fmul_rn(v.lo, scale));  // |L| <= 2^29
  const int64_t delta = (hb >> 31) ? -(int64_t)L : (int64_t)L;  // in magnitude units
  const uint64_t mag = (((uint64_t)(e8 + 896u) << 52) | ((uint64_t)mant << 29)) + (uint64_t)delta;
  return __longlong_as_double((long long)(((uint64_t)(hb >> 31) << 63) | mag));
}

// AccurateDWPlusDW (Joldes et al. 2017, Alg. 6): relative error <= 3u^2
TE_DEV dw dw_add(dw x, dw y) {
  float sh, sl, th, tl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  float c = __fadd_rn(sl, th);
  float vh, vl;
  fast_two_sum(sh, c, vh, vl);
  float w = __fadd_rn(tl, vl);
  dw z;
  fast_two_sum(vh, w, z.hi, z.lo);
  return z;
}
TE_DEV dw dw_neg(dw x) { return dw{-x.hi, -x.lo}; }
TE_DEV dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

// DWTimesDW (Joldes et al. 2017, Alg. 10 style, FMA based)
TE_DEV dw dw_mul(dw x, dw y) {
  float ch, cl1;
  two_prod(x.hi, y.hi, ch, cl1);
  float tl = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
  float cl2 = __fadd_rn(cl1, tl);
  dw z;
  fast_two_sum(ch, cl2, z.hi, z.lo);
  return z;
}

// ---------------------------------------------------------------------------
// compensated accumulator (Dot2 of Ogita, Rump & Oishi): value = s + c
// ---------------------------------------------------------------------------
struct dacc {
  float s, c;
};
TE_DEV dacc dacc_zero() { return dacc{0.f, 0.f}; }
// acc += x * (yh + yl), the product x*yh taken exactly
TE_DEV void dacc_fma(dacc& a, float x, float yh, float yl) {
  float p, ep;
  two_prod(x, yh, p, ep);
  float s, es;
  two_sum(a.s, p, s, es);
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(es, __fmaf_rn(x, yl, ep)));
}
// acc += (p + e) where p + e is an exact product pair
TE_DEV void dacc_add_pair(dacc& a, float p, float e) {
  float s, es;
  two_sum(a.s, p, s, es);
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(es, e));
}
TE_DEV void dacc_add_dw(dacc& a, dw v) { dacc_add_pair(a, v.hi, v.lo); }
TE_DEV dacc dacc_merge(dacc a, dacc b) {
  float s, es;
  two_sum(a.s, b.s, s, es);
  return dacc{s, __fadd_rn(__fadd_rn(a.c, b.c), es)};
}
TE_DEV dw dacc_value(dacc a) {
  dw z;
  two_sum(a.s, a.c, z.hi, z.lo);
  return z;
}

// ---------------------------------------------------------------------------
// warp reductions (fixed xor tree: deterministic)
// ---------------------------------------------------------------------------
TE_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
TE_DEV dacc warp_sum(dacc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dacc w;
    w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
    w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
    v = dacc_merge(v, w);
  }
  return v;
}
// reduce within aligned groups of `width` lanes (width a power of two <= 32)
TE_DEV double group_sum(double v, int width) {
  for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
TE_DEV dacc group_sum(dacc v, int width) {
  for (int o = width >> 1; o > 0; o >>= 1) {
    dacc w;
    w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
    w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
    v = dacc_merge(v, w);
  }
  return v;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), addressed by
// (seed, stream, index): i-th output of the generator whose state starts at
// seed XOR stream*0xD1B54A32D192ED03.  uniform(-1,1) = 2*(x>>11)*2^-53 - 1.
// ---------------------------------------------------------------------------
TE_DEV uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
TE_DEV double sm64_uniform_pm1(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t s0 = seed ^ (stream * 0xD1B54A32D192ED03ULL);
  uint64_t x = sm64_mix(s0 + (i + 1) * 0x9E3779B97F4A7C15ULL);
  return 2.0 * ((double)(x >> 11) * 0x1.0p-53) - 1.0;
}

// ---------------------------------------------------------------------------
// memory-access helpers
// ---------------------------------------------------------------------------
TE_DEV uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
TE_DEV uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// gathers of the SpMV's x: read-only, kept in L2 ahead of the streamed layout
TE_DEV float ld_keep_f32(const float* a, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
TE_DEV double ld_keep_f64(const double* a, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
// a gather issued only where `on` is set (predicated: a warp's gathers stay in
// flight together), allocating in L1 or not; 0 elsewhere
template <bool ALLOC>
TE_DEV float ld_keep_f32_if(const float* a, bool on, uint64_t pol) {
  float v = 0.f;
  if constexpr (ALLOC)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n"
        " @p ld.global.nc.L2::cache_hint.f32 %0, [%1], %3;\n}"
        : "+f"(v) : "l"(a), "r"((unsigned)on), "l"(pol));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n"
        " @p ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %3;\n}"
        : "+f"(v) : "l"(a), "r"((unsigned)on), "l"(pol));
  return v;
}
template <bool ALLOC>
TE_DEV double ld_keep_f64_if(const double* a, bool on, uint64_t pol) {
  double v = 0.0;
  if constexpr (ALLOC)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n"
        " @p ld.global.nc.L2::cache_hint.f64 %0, [%1], %3;\n}"
        : "+d"(v) : "l"(a), "r"((unsigned)on), "l"(pol));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n"
        " @p ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %3;\n}"
        : "+d"(v) : "l"(a), "r"((unsigned)on), "l"(pol));
  return v;
}
TE_DEV int ld_stream_i32(const int32_t* a, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
               : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
TE_DEV float ld_stream_f32(const float* a, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
TE_DEV uint32_t ld_stream_u16(const uint16_t* a, uint64_t pol) {
  unsigned short v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;"
               : "=h"(v) : "l"(a), "l"(pol));
  return v;
}
TE_DEV uint32_t ld_stream_u8(const uint8_t* a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u8 %0, [%1], %2;"
               : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
// reduced-precision matrix values -> binary32 (exact)
TE_DEV float bf16_to_f32(uint32_t code) { return __uint_as_float(code << 16); }
// FP8 E4M3 (sign, 4 exponent bits with bias 7, 3 fraction bits; exponent 0
// subnormal) -> binary32 by the hardware conversion to half precision, which
// is exact for every finite E4M3 value, then half -> binary32 (exact).  The
// code is placed in both bytes of the converted pair, so either half holds it.
TE_DEV float e4m3_to_f32(uint32_t code) {
  const unsigned short pair = (unsigned short)((code & 0xffu) * 0x0101u);
  uint32_t h2;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(pair));
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"((unsigned short)(h2 & 0xffffu)));
  return f;
}
TE_DEV double ld_stream_f64(const double* a, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
               : "=d"(v) : "l"(a), "l"(pol));
  return v;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (TMA, non-tensor form) wrappers
// ---------------------------------------------------------------------------
TE_DEV uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
TE_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
TE_DEV void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
TE_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
TE_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
TE_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: returns false after `limit` unsuccessful polls (each poll may
// itself suspend for a hardware-defined time).
TE_DEV bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy, completion signalled on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned)
TE_DEV void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar,
                     uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_addr(dst_smem)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
TE_DEV void named_bar_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

}  // namespace te
