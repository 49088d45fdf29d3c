// peak.cu -- arithmetic peak rates of this GPU, measured by the library itself (the ALU
// roofline denominators of the measurement helpers): FP32 FMA, FP64 FMA and the lazy
// float-float multiply-add that the float-float kernels use for their dot products.
//
// Every thread runs NCH independent multiply-add chains in registers (enough to cover the
// pipeline latency), for `iters` steps, and writes one value so that nothing is removed as
// dead code.  The grid fills every SM (8 CTAs of 256 threads each).
#include "arith.cuh"
#include "engine.h"
#include "tt_svd.h"

namespace tt {
namespace {

constexpr int NCH = 8;

// written only in a case that does not occur (keeps the chains from being removed)
__device__ double g_sink[1];

template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T a, T b, T* out) {
  T x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fmac(x[c], a, b);
  T s = x[0];
#pragma unroll
  for (int c = 1; c < NCH; ++c) s = s + x[c];
  if (s == (T)-1) out[0] = s;  // practically never: keeps the chains alive
}

// float-float: acc + a*b with the lazy accumulator (lz_fmac, 12 FP32 instructions), the
// form of the float-float dot products; one step counts as one FP64-equivalent FMA
__global__ void __launch_bounds__(256) k_df_rate(int iters, df a, float* out) {
  dfl x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) { x[c].s = (float)(threadIdx.x + c) * 1e-3f; x[c].e = 0.f; }
  df w = mkdf(1.0f + threadIdx.x * 1e-7f, 0.f);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = lz_fmac(a, w, x[c]);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c].s + x[c].e;
  if (s == -1.f) out[0] = s;
}

// FP64 tensor-core MMA (mma.sync m8n8k4, f64 in and out): NCH independent accumulator
// tiles per warp; one MMA is 8 x 8 x 4 multiply-adds
__global__ void __launch_bounds__(256) k_dmma_rate(int iters, double a0, double* out) {
  double acc[NCH][2];
#pragma unroll
  for (int c = 0; c < NCH; ++c) { acc[c][0] = 0.0; acc[c][1] = 0.0; }
  const double a = a0 + threadIdx.x * 1e-9, b = 1e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < NCH; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += acc[c][0] + acc[c][1];
  if (s == -1.0) out[0] = s;
}

}  // namespace
}  // namespace tt

using namespace tt;

extern "C" tt_status tt_fma_rate(int kind, double* flops_per_s, void* stream) {
  if (!flops_per_s || kind < 0 || kind > 3) return TT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)num_sms() * 8;
  // enough steps for ~50-100 ms of work at the expected rates
  const int iters = kind == 1 ? 2048 : (kind == 0 ? 131072 : (kind == 2 ? 16384 : 256));
  void* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  tt_status st = TT_OK;
  if (cudaGetSymbolAddress(&out, g_sink) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    st = TT_ECUDA;
  } else {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && st == TT_OK; ++rep) {  // the first run is a warm-up
      cudaEventRecord(a, s);
      if (kind == 0) k_fma_rate<float><<<grid, 256, 0, s>>>(iters, 0.999f, 1e-4f, (float*)out);
      else if (kind == 1) k_fma_rate<double><<<grid, 256, 0, s>>>(iters, 0.999, 1e-4, (double*)out);
      else if (kind == 2) k_df_rate<<<grid, 256, 0, s>>>(iters, df{0.999f, 1e-9f}, (float*)out);
      else k_dmma_rate<<<grid, 256, 0, s>>>(iters, 0.999, (double*)out);
      cudaEventRecord(b, s);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&ms, a, b) != cudaSuccess || !(ms > 0.f))
        st = TT_ECUDA;
    }
    // multiply-adds per launch: one per thread, chain and step (FMA kinds); one MMA per
    // warp, chain and step is 8 x 8 x 4 of them (kind 3)
    const double madds = kind == 3 ? (double)grid * 8.0 * NCH * iters * 256.0
                                   : (double)grid * 256.0 * NCH * (double)iters;
    if (st == TT_OK) *flops_per_s = 2.0 * madds / (ms * 1e-3);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st != TT_OK) set_last_error_text("tt_fma_rate: a CUDA call failed");
  return st;
}
