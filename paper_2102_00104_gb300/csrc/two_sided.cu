// two_sided.cu -- kernels of the two-sided TT-SVD (Alg. 4, Sec. 3.1.3): the transposes
// between right and left steps, the cores of a left and of a right step, the
// discarded energy and the ranks.  The steps themselves reuse the TSQR, Jacobi and
// W*V_r kernels (driver.cu plans and queues them).
#include <cstdint>

#include "tsqr_kernels.cuh"

namespace tt {

namespace {

// out (Q x P, column-major) = in (P x Q, column-major)^T, 32 x 32 tiles through shared
// memory so that both the reads and the writes are coalesced; a grid-stride loop over
// the tiles (either extent may be large)
template <class T>
__global__ void __launch_bounds__(256) k_transpose(const T* __restrict__ in, int64_t P, int64_t Q,
                                                   T* __restrict__ out) {
  __shared__ T tile[32][33];
  const int64_t tp = (P + 31) / 32, tq = (Q + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int64_t t = blockIdx.x; t < tp * tq; t += gridDim.x) {
    const int64_t p0 = (t % tp) * 32, q0 = (t / tp) * 32;
    for (int j = ty; j < 32; j += 8) {
      const int64_t p = p0 + tx, q = q0 + j;
      if (p < P && q < Q) tile[j][tx] = in[p + P * q];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
      const int64_t q = q0 + tx, p = p0 + j;
      if (p < P && q < Q) out[q + Q * p] = tile[tx][j];
    }
    __syncthreads();
  }
}

// right step: T (r x m, the (r_{i-1}) x (n_i r_i) matricization) = V_{:,1:r}^T
template <class C>
__global__ void k_core_right(const C* __restrict__ V, int ldV, int m, int r, double* __restrict__ core) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % r), j = (int)(idx / r);
    core[idx] = to_f64(V[j + (size_t)a * ldV]);
  }
}

// left step: T (m x r, the (r_{i-1} n_i) x r_i matricization) = V_{:,1:r}
template <class C>
__global__ void k_core_left(const C* __restrict__ V, int ldV, int m, int r, double* __restrict__ core) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % m), a = (int)(idx / m);
    core[idx] = to_f64(V[j + (size_t)a * ldV]);
  }
}

// e += sum_{k = r}^{cnt-1} sigma_k^2 (sigma sorted descending)
__global__ void k_add_discarded(const double* __restrict__ sigma, int cnt, int r, double* e) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = r; k < cnt; ++k) s = fma(sigma[k], sigma[k], s);
  *e += s;
}

struct RankList {
  int64_t r[TT_MAX_RANKS];
};

__global__ void k_put_ranks(RankList rl, int count, int64_t* ranks_out, const double* e,
                            double* err2_out, const XRange* xr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ranks_out)
    for (int i = 0; i < count; ++i) ranks_out[i] = rl.r[i];
  // the discarded sigma^2 were of X 2^-k
  if (err2_out) *err2_out = xr ? ldexp(*e, 2 * xr->k) : *e;
}

__global__ void k_zero(double* e) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *e = 0.0;
}

unsigned grid_of(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 65536) g = 65536;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_transpose(size_t elem, const void* in, int64_t P, int64_t Q, void* out,
                             cudaStream_t s) {
  const int64_t tiles = ((P + 31) / 32) * ((Q + 31) / 32);
  const unsigned g = (unsigned)std::min<int64_t>(std::max<int64_t>(tiles, 1), 152 * 16);
  if (elem == 8)
    k_transpose<uint64_t><<<g, 256, 0, s>>>(static_cast<const uint64_t*>(in), P, Q, static_cast<uint64_t*>(out));
  else if (elem == 4)
    k_transpose<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(in), P, Q, static_cast<uint32_t*>(out));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_core_side(Fmt vfmt, bool left, const void* V, int ldV, int m, int r, double* core,
                             cudaStream_t s) {
  const unsigned g = grid_of((int64_t)m * r, 256);
  if (vfmt == Fmt::DF) {
    if (left) k_core_left<df><<<g, 256, 0, s>>>(static_cast<const df*>(V), ldV, m, r, core);
    else k_core_right<df><<<g, 256, 0, s>>>(static_cast<const df*>(V), ldV, m, r, core);
  } else if (vfmt == Fmt::F64) {
    if (left) k_core_left<double><<<g, 256, 0, s>>>(static_cast<const double*>(V), ldV, m, r, core);
    else k_core_right<double><<<g, 256, 0, s>>>(static_cast<const double*>(V), ldV, m, r, core);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_add_discarded(const double* sigma, int cnt, int r, double* e, cudaStream_t s) {
  k_add_discarded<<<1, 32, 0, s>>>(sigma, cnt, r, e);
  return cudaGetLastError();
}

cudaError_t launch_zero(double* e, cudaStream_t s) {
  k_zero<<<1, 32, 0, s>>>(e);
  return cudaGetLastError();
}

cudaError_t launch_put_ranks(const int64_t* ranks, int count, int64_t* ranks_out, const double* e,
                             double* err2_out, cudaStream_t s, const XRange* xr) {
  if (count > TT_MAX_RANKS) return cudaErrorInvalidValue;
  RankList rl{};
  for (int i = 0; i < count; ++i) rl.r[i] = ranks[i];
  k_put_ranks<<<1, 32, 0, s>>>(rl, count, ranks_out, e, err2_out, xr);
  return cudaGetLastError();
}

}  // namespace tt
