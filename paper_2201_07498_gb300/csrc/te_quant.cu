// te_quant.cu - rounding of binary64 matrix values to the storage types of
// the mixed-precision forms (Section III-A): binary32, bfloat16, and FP8 E4M3
// with one binary32 scale per row.
//
// Round to nearest, ties to even, from the binary64 value directly (no
// intermediate binary32 rounding); a zero result is +0.  For |x| in
// [2^e, 2^(e+1)) and p significant bits the quantum is 2^(e+1-p), never below
// the format's smallest subnormal; |x| / quantum is exact and rint() rounds
// it to the nearest integer, ties to even.  FP8: scale_r = binary32 of
// max_j |a_rj| / 448 (1 for an all-zero row), code = round(a / scale_r)
// saturated at 448 (the largest finite E4M3 value).
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

TE_DEV double round_sig(double ax, int p, int qmin) {
  int qe = ilogb(ax) + 1 - p;
  if (qe < qmin) qe = qmin;
  const double q = scalbn(1.0, qe);
  return rint(ax / q) * q;
}

TE_DEV uint16_t bf16_code(double x) {
  const double ax = fabs(x);
  if (!(ax > 0.0)) return 0;
  const double r = round_sig(ax, 8, -133);
  if (r == 0.0) return 0;
  const uint32_t bits = __float_as_uint((float)r);  // exact: 8 significant bits
  return (uint16_t)((bits >> 16) | (x < 0.0 ? 0x8000u : 0u));
}

TE_DEV uint8_t e4m3_code(double x) {
  const double ax = fabs(x);
  if (!(ax > 0.0)) return 0;
  double r = round_sig(ax, 4, -9);
  if (r > 448.0) r = 448.0;
  if (r == 0.0) return 0;
  uint32_t code;
  if (r < 0x1p-6) {
    code = (uint32_t)(r * 512.0);  // subnormal: m * 2^-9, m in 1..7
  } else {
    const int e = ilogb(r);
    code = ((uint32_t)(e + 7) << 3) | ((uint32_t)scalbn(r, 3 - e) - 8u);
  }
  return (uint8_t)(code | (x < 0.0 ? 0x80u : 0u));
}

__global__ void round_f32_kernel(const double* v, int64_t nnz, float* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = __double2float_rn(v[k]);
}

__global__ void round_bf16_kernel(const double* v, int64_t nnz, uint16_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = bf16_code(v[k]);
}

// one warp per row: the row's largest magnitude gives its scale
__global__ void quant_e4m3_kernel(const int64_t* rp, const double* v, int64_t n, uint8_t* out,
                                  float* scale) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t a = rp[r], b = rp[r + 1];
    double mx = 0.0;
    for (int64_t k = a + lane; k < b; k += 32) mx = fmax(mx, fabs(v[k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = mx > 0.0 ? __double2float_rn(mx / 448.0) : 1.0f;
    if (lane == 0) scale[r] = s;
    for (int64_t k = a + lane; k < b; k += 32) out[k] = e4m3_code(v[k] / (double)s);
  }
}

cudaError_t launch_quantize(int to, const int64_t* rp, const double* val, int64_t n, int64_t nnz,
                            void* out, float* row_scale, cudaStream_t s) {
  const int threads = 256;
  if (to == TE_FP8_E4M3) {
    int64_t blocks = (n * 32 + threads - 1) / threads;
    if (blocks > 65536) blocks = 65536;
    if (blocks < 1) blocks = 1;
    quant_e4m3_kernel<<<(int)blocks, threads, 0, s>>>(rp, val, n, static_cast<uint8_t*>(out),
                                                       row_scale);
    return cudaGetLastError();
  }
  if (nnz <= 0) return cudaSuccess;
  int64_t blocks = (nnz + threads - 1) / threads;
  if (blocks > 65536) blocks = 65536;
  if (to == TE_BF16)
    round_bf16_kernel<<<(int)blocks, threads, 0, s>>>(val, nnz, static_cast<uint16_t*>(out));
  else if (to == TE_F32)
    round_f32_kernel<<<(int)blocks, threads, 0, s>>>(val, nnz, static_cast<float*>(out));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace te
