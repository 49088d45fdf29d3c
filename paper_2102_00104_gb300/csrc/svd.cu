// svd.cu -- small SVD of R (Eq. QR_trick), the rank choice (Alg. 2 lines 7-8),
// the core write (line 9), the last core (line 13) and small helpers.
//
// The SVD is one-sided Jacobi (Hestenes): columns of A = R are rotated in
// pairs until they are mutually orthogonal; then sigma_j = ||a_j|| and the
// accumulated rotations form V.  It works on R itself (never on R^T R), so
// small singular values keep their accuracy.  Pairs follow the round-robin
// (circle) ordering: m-1 rounds of m/2 disjoint pairs per sweep, one group of
// 8-32 lanes per pair.  The rotation angle is taken from zeta = (beta - alpha) / (2 gamma)
// with t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) (the 2x2 symmetric Schur
// decomposition of [[alpha, gamma], [gamma, beta]]); beta - alpha is formed in
// the working arithmetic, zeta and t in FP32, and c = 1/sqrt(1+t^2), s = c t in
// the working arithmetic, so each rotation is orthogonal to working precision
// even though its angle is only FP32-accurate (the next sweep removes the
// remaining small coupling).
#include <cstdio>
#include <mutex>

#include "tsqr_col.cuh"
#include "tt_svd.h"

namespace tt {

namespace {

__device__ __forceinline__ float fp32_hi(df a) { return a.hi; }
__device__ __forceinline__ float fp32_hi(double a) { return (float)a; }
__device__ __forceinline__ float fp32_hi(float a) { return a; }

template <class C> __device__ __forceinline__ C scale_pow2(C a, int e);
template <> __device__ __forceinline__ df scale_pow2<df>(df a, int e) {
  return mkdf(ldexpf(a.hi, e), ldexpf(a.lo, e));
}
template <> __device__ __forceinline__ double scale_pow2<double>(double a, int e) { return ldexp(a, e); }

template <class C> __device__ __forceinline__ C from_f32(float x);
template <> __device__ __forceinline__ df from_f32<df>(float x) { return mkdf(x, 0.f); }
template <> __device__ __forceinline__ double from_f32<double>(float x) { return (double)x; }

// Rotation threshold on |cos(a_p, a_q)|: above the rounding floor of an m-term
// dot product in the working arithmetic (unit roundoff ~2^-46 for the sloppy
// float-float operations, 2^-53 for FP64), so the sweeps terminate.
template <class C> __device__ __forceinline__ float conv_tol(int m);
template <> __device__ __forceinline__ float conv_tol<df>(int m) { return 2.0e-14f * (float)(m < 8 ? 8 : m); }
template <> __device__ __forceinline__ float conv_tol<double>(int m) { return 2.5e-16f * (float)(m < 8 ? 8 : m); }

// float-float (or FP64) rotation parameters from an FP32-accurate tangent t:
// c = 1 / sqrt(1 + t^2) to working precision (two Newton steps c <- c + c (1 - u c^2) / 2
// from the FP32 reciprocal square root), s = c t, so c^2 + s^2 = 1 to working precision.
__device__ __forceinline__ void rot_cs(float t, df& c, df& sn) {
  float p, e;
  eft_two_prod(t, t, p, e);
  const df u = add(mkdf(1.f, 0.f), mkdf(p, e));       // 1 + t^2, exact up to df rounding
  df cc = mkdf(rsqrtf(u.hi), 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df r = fnmac(u, mul(cc, cc), mkdf(1.f, 0.f));  // 1 - u c^2
    cc = fmac(mul(cc, mkdf(0.5f, 0.f)), r, cc);
  }
  c = cc;
  sn = mul(cc, mkdf(t, 0.f));
}
__device__ __forceinline__ void rot_cs(float t, double& c, double& sn) {
  c = 1.0 / sqrt(1.0 + (double)t * (double)t);
  sn = c * (double)t;
}

// masked butterfly inside a group of G lanes (G divides 32, groups are aligned)
template <int G>
__device__ __forceinline__ df gsum(df a, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
    a = add(a, mkdf(__shfl_xor_sync(mask, a.hi, o), __shfl_xor_sync(mask, a.lo, o)));
  return a;
}
template <int G>
__device__ __forceinline__ double gsum(double a, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(mask, a, o);
  return a;
}

// One thread block; A, V in shared memory when `smem_ok`, else in global (Ag, Vg).
// Each pair (p, q) of a round is handled by a group of G lanes.
template <class C, class RI, int G>
__global__ void __launch_bounds__(1024)
k_jacobi(const RI* __restrict__ R, int64_t ldR, const int* __restrict__ m_ptr, int m_max,
         C* __restrict__ Ag, C* __restrict__ Vg, int ldA, int smem_ok, double* __restrict__ sigma,
         C* __restrict__ Vout, int ldV, int* status, int* sweeps_out, int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  __shared__ int s_exp;
  __shared__ float s_red[32];
  const int m = m_ptr ? *m_ptr : m_max;
  if (m < 1 || m > m_max) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int mp = m + (m & 1);  // even count of columns (one zero column added for odd m)
  C* A = smem_ok ? reinterpret_cast<C*>(smem_raw) : Ag;
  C* V = smem_ok ? reinterpret_cast<C*>(smem_raw) + (size_t)ldA * mp : Vg;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nt >> 5;

  // exponent of max |R| for an exact power-of-two scaling (keeps squares in FP32 range)
  float mx = 0.f;
  for (int idx = tid; idx < m * m; idx += nt) {
    const int i = idx % m, k = idx / m;
    const float v = fabsf(fp32_hi(ld_as<C>(R[i + (int64_t)k * ldR])));
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarps; ++w) t = fmaxf(t, s_red[w]);
    int e = 0;
    if (t > 0.f) frexpf(t, &e);
    s_exp = e;
  }
  __syncthreads();
  const int ex = s_exp;
  for (int idx = tid; idx < ldA * mp; idx += nt) {
    const int i = idx % ldA, k = idx / ldA;
    C a = Tr<C>::zero();
    if (i < m && k < m && i <= k) a = flush_tiny(scale_pow2<C>(ld_as<C>(R[i + (int64_t)k * ldR]), -ex));
    A[idx] = a;
    V[idx] = (i == k) ? Tr<C>::one() : Tr<C>::zero();
  }
  __syncthreads();

  // ||A||_F^2 (FP32 is enough): pairs whose norm product is below tol^2 ||A||_F^2
  // consist of rounding noise (rank-deficient R) and are not rotated, otherwise
  // such columns would keep coupling with each other and never converge
  float fro = 0.f;
  for (int idx = tid; idx < ldA * mp; idx += nt) {
    const float v = fp32_hi(A[idx]);
    fro = fmaf(v, v, fro);
  }
  for (int o = 16; o; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  __syncthreads();
  if (lane == 0) s_red[wid] = fro;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarps; ++w) t += s_red[w];
    s_red[0] = t;
  }
  __syncthreads();
  const float tol = conv_tol<C>(m);
  const float floor_abs = tol * tol * s_red[0];
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));

  __shared__ int s_cos;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s_rot = 0;
      s_cos = 0;
    }
    __syncthreads();
    bool rot_t = false;   // this thread's rotations and largest |cos|, combined per sweep
    float mcos_t = 0.f;
    for (int rnd = 0; rnd < mp - 1; ++rnd) {
      for (int slot = gid; slot < mp / 2; slot += ngroups) {
        int p, q;
        if (slot == 0) {
          p = mp - 1;
          q = rnd;
        } else {
          p = (rnd + slot) % (mp - 1);
          q = (rnd - slot + mp - 1) % (mp - 1);
        }
        C* ap = A + (size_t)p * ldA;
        C* aq = A + (size_t)q * ldA;
        auto al = lz(Tr<C>::zero()), be = al, ga = al;  // lazy float-float sums
        for (int i = gl; i < m; i += G) {
          const C x = ap[i], y = aq[i];
          al = lz_fmac(x, x, al);
          be = lz_fmac(y, y, be);
          ga = lz_fmac(x, y, ga);
        }
        const C alf = lz_fin(lz_gsum<G>(al, gmask));
        const C bef = lz_fin(lz_gsum<G>(be, gmask));
        const C gaf = lz_fin(lz_gsum<G>(ga, gmask));
        const float gf = fabsf(fp32_hi(gaf));
        const float nf = sqrtf(fp32_hi(alf)) * sqrtf(fp32_hi(bef));
        if (gf > tol * nf && nf > floor_abs && gf > 0.f) {
          // zeta = (beta - alpha) / (2 gamma): difference in working precision, quotient in FP32
          const float zf = fp32_hi(sub(bef, alf)) / (2.f * fp32_hi(gaf));
          const float az = fabsf(zf);
          float tf = az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f)));
          if (zf < 0.f) tf = -tf;
          C c, s;
          rot_cs(tf, c, s);
          for (int i = gl; i < m; i += G) {
            const C x = ap[i], y = aq[i];
            ap[i] = fnmac(s, y, mul(c, x));
            aq[i] = fmac(s, x, mul(c, y));
          }
          C* vp = V + (size_t)p * ldA;
          C* vq = V + (size_t)q * ldA;
          for (int i = gl; i < mp; i += G) {
            const C x = vp[i], y = vq[i];
            vp[i] = fnmac(s, y, mul(c, x));
            vq[i] = fmac(s, x, mul(c, y));
          }
          rot_t = true;
          mcos_t = fmaxf(mcos_t, gf / nf);
        }
      }
      __syncthreads();
    }
    const bool any_w = __any_sync(0xffffffffu, rot_t);
    for (int o = 16; o; o >>= 1) mcos_t = fmaxf(mcos_t, __shfl_xor_sync(0xffffffffu, mcos_t, o));
    if (lane == 0 && any_w) {
      s_rot = 1;
      atomicMax(&s_cos, __float_as_int(mcos_t));  // |cos| >= 0: int order = float order
    }
    __syncthreads();
    // converged when nothing rotated, or when every rotation of the sweep had |cos| < 1e-7
    // (the coupling left after it is of the order of those squared)
    if (s_rot == 0 || __int_as_float(s_cos) < 1e-7f) break;
    __syncthreads();
  }
  if (sweep >= max_sweeps && tid == 0 && status) atomicOr(status, DEV_SVD_NOCONV);
  if (tid == 0 && sweeps_out) *sweeps_out = sweep + 1;

  // sigma_k = ||a_k||, sorted descending (stable by index); V columns follow
  C* nrm = smem_ok ? V + (size_t)ldA * mp : reinterpret_cast<C*>(smem_raw);
  for (int k = tid; k < m; k += nt) {
    C nk = Tr<C>::zero();
    const C* ak = A + (size_t)k * ldA;
    for (int i = 0; i < m; ++i) nk = fmac(ak[i], ak[i], nk);
    nrm[k] = nk;
  }
  __syncthreads();
  for (int k = tid; k < m; k += nt) {
    const C nk = nrm[k];
    int rank = 0;
    for (int k2 = 0; k2 < m; ++k2) {
      if (k2 == k) continue;
      const C n2 = nrm[k2];
      if (is_gt(n2, nk) || (!is_gt(nk, n2) && k2 < k)) ++rank;
    }
    const double sg = ldexp(to_f64(sqrt_(nk)), ex);
    if (!isfinite(sg) && status) atomicOr(status, DEV_NONFINITE);
    sigma[rank] = sg;
    const C* vk = V + (size_t)k * ldA;
    for (int i = 0; i < m; ++i) Vout[i + (size_t)rank * ldV] = vk[i];
  }
}

// ---- wide unfoldings (rows < columns) ---------------------------------------------
// For W (rows x m) with rows < m the R of Alg. 2 has only `rows` nonzero rows, so its SVD
// is that of W itself (a zero-padded R has the same nonzero sigma and V).  One-sided
// Jacobi on the `rows` columns of A = W^T (each of length m) takes (rows/m)^2 of the
// column pairs of the square form and accumulates nothing: at convergence the columns
// are sigma_k v_k, so v_k = a_k / ||a_k||.  Columns at the rounding floor (the ones the
// sweeps leave unrotated, see k_jacobi) and zero columns get an orthonormal completion
// instead: unit vectors, Gram-Schmidt twice against the columns before them.
template <class C, class WI, int G>
__global__ void __launch_bounds__(1024)
k_jacobi_wide(const WI* __restrict__ W, int64_t ldW, int rows, const int* __restrict__ m_ptr,
              int m_max, int lda, double* __restrict__ sigma, C* __restrict__ Vout, int ldV,
              int* status, int* sweeps_out, int max_sweeps, C* __restrict__ Aglob) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  __shared__ int s_cos;
  __shared__ int s_exp;
  __shared__ float s_red[32];
  const int m = m_ptr ? *m_ptr : m_max;
  const int nc = rows, ncp = rows + (rows & 1);
  if (m < 1 || m > m_max || m > lda || nc < 1) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  // column p (= row p of W) at A + p * lda: in shared memory, or (when rows x m does not
  // fit there) in an L2-resident global scratch that only this CTA touches
  C* A = Aglob ? Aglob : reinterpret_cast<C*>(smem_raw);
  C* nrm = Aglob ? reinterpret_cast<C*>(smem_raw) : A + (size_t)ncp * lda;  // ||a_k||^2
  int* defi = reinterpret_cast<int*>(nrm + ncp);  // by rank: 1 = completion needed
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nt >> 5;

  float mx = 0.f;
  for (int idx = tid; idx < nc * m; idx += nt) {
    const int p = idx % nc, i = idx / nc;
    mx = fmaxf(mx, fabsf(fp32_hi(ld_as<C>(W[p + (int64_t)i * ldW]))));
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarps; ++w) t = fmaxf(t, s_red[w]);
    int e = 0;
    if (t > 0.f) frexpf(t, &e);
    s_exp = e;
  }
  __syncthreads();
  const int ex = s_exp;
  for (int idx = tid; idx < ncp * m; idx += nt) {
    const int p = idx % ncp, i = idx / ncp;
    A[i + (size_t)p * lda] =
        p < nc ? flush_tiny(scale_pow2<C>(ld_as<C>(W[p + (int64_t)i * ldW]), -ex)) : Tr<C>::zero();
  }
  __syncthreads();
  float fro = 0.f;
  for (int idx = tid; idx < ncp * m; idx += nt) {
    const float v = fp32_hi(A[(idx % m) + (size_t)(idx / m) * lda]);
    fro = fmaf(v, v, fro);
  }
  for (int o = 16; o; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if (lane == 0) s_red[wid] = fro;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < nwarps; ++w) t += s_red[w];
    s_red[0] = t;
  }
  __syncthreads();
  const float tol = conv_tol<C>(m);
  const float floor_abs = tol * tol * s_red[0];
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s_rot = 0;
      s_cos = 0;
    }
    __syncthreads();
    bool rot_t = false;   // this thread's rotations and largest |cos|, combined per sweep
    float mcos_t = 0.f;
    for (int rnd = 0; rnd < ncp - 1; ++rnd) {
      for (int slot = gid; slot < ncp / 2; slot += ngroups) {
        int p, q;
        if (slot == 0) {
          p = ncp - 1;
          q = rnd;
        } else {
          p = (rnd + slot) % (ncp - 1);
          q = (rnd - slot + ncp - 1) % (ncp - 1);
        }
        C* ap = A + (size_t)p * lda;
        C* aq = A + (size_t)q * lda;
        auto al = lz(Tr<C>::zero()), be = al, ga = al;
        for (int i = gl; i < m; i += G) {
          const C x = ap[i], y = aq[i];
          al = lz_fmac(x, x, al);
          be = lz_fmac(y, y, be);
          ga = lz_fmac(x, y, ga);
        }
        const C alf = lz_fin(lz_gsum<G>(al, gmask));
        const C bef = lz_fin(lz_gsum<G>(be, gmask));
        const C gaf = lz_fin(lz_gsum<G>(ga, gmask));
        const float gf = fabsf(fp32_hi(gaf));
        const float nf = sqrtf(fp32_hi(alf)) * sqrtf(fp32_hi(bef));
        if (gf > tol * nf && nf > floor_abs && gf > 0.f) {
          const float zf = fp32_hi(sub(bef, alf)) / (2.f * fp32_hi(gaf));
          const float az = fabsf(zf);
          float tf = az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f)));
          if (zf < 0.f) tf = -tf;
          C c, s;
          rot_cs(tf, c, s);
          for (int i = gl; i < m; i += G) {
            const C x = ap[i], y = aq[i];
            ap[i] = fnmac(s, y, mul(c, x));
            aq[i] = fmac(s, x, mul(c, y));
          }
          rot_t = true;
          mcos_t = fmaxf(mcos_t, gf / nf);
        }
      }
      __syncthreads();
    }
    const bool any_w = __any_sync(0xffffffffu, rot_t);
    for (int o = 16; o; o >>= 1) mcos_t = fmaxf(mcos_t, __shfl_xor_sync(0xffffffffu, mcos_t, o));
    if (lane == 0 && any_w) {
      s_rot = 1;
      atomicMax(&s_cos, __float_as_int(mcos_t));
    }
    __syncthreads();
    if (s_rot == 0 || __int_as_float(s_cos) < 1e-7f) break;
    __syncthreads();
  }
  if (sweep >= max_sweeps && tid == 0 && status) atomicOr(status, DEV_SVD_NOCONV);
  if (tid == 0 && sweeps_out) *sweeps_out = sweep + 1;

  // sigma_k = ||a_k||, descending (stable by index); v_k = a_k / ||a_k||
  for (int k = tid; k < nc; k += nt) {
    auto acc = lz(Tr<C>::zero());
    const C* ak = A + (size_t)k * lda;
    for (int i = 0; i < m; ++i) acc = lz_fmac(ak[i], ak[i], acc);
    nrm[k] = lz_fin(acc);
  }
  __syncthreads();
  const int nout = nc < m ? nc : m;
  for (int k = tid; k < nc; k += nt) {
    const C nk = nrm[k];
    int rank = 0;
    for (int k2 = 0; k2 < nc; ++k2) {
      if (k2 == k) continue;
      const C n2 = nrm[k2];
      if (is_gt(n2, nk) || (!is_gt(nk, n2) && k2 < k)) ++rank;
    }
    if (rank >= nout) continue;
    const C sk = sqrt_(nk);
    const double sg = ldexp(to_f64(sk), ex);
    if (!isfinite(sg) && status) atomicOr(status, DEV_NONFINITE);
    sigma[rank] = sg;
    const bool low = !(fp32_hi(nk) > floor_abs);
    defi[rank] = low ? 1 : 0;
    if (!low) {
      const C inv = rcp_(sk);
      const C* ak = A + (size_t)k * lda;
      for (int i = 0; i < m; ++i) Vout[i + (size_t)rank * ldV] = mul(ak[i], inv);
    }
  }
  __syncthreads();
  // completion of the columns at the rounding floor (they have the largest ranks)
  if (wid != 0) return;
  constexpr int QV = kMaxM / 32;
  int cand = 0;
  for (int p = 0; p < nout; ++p) {
    if (!defi[p]) continue;
    for (; cand < m; ++cand) {
      C v[QV];
#pragma unroll
      for (int u = 0; u < QV; ++u)
        v[u] = (lane + 32 * u == cand) ? Tr<C>::one() : Tr<C>::zero();
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = 0; q < p; ++q) {
          const C* vq = Vout + (size_t)q * ldV;
          auto acc = lz(Tr<C>::zero());
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const int i = lane + 32 * u;
            if (i < m) acc = lz_fmac(vq[i], v[u], acc);
          }
          const C h = colk::warp_allsum(lz_fin(acc));
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const int i = lane + 32 * u;
            if (i < m) v[u] = fnmac(h, vq[i], v[u]);
          }
        }
      }
      auto acc = lz(Tr<C>::zero());
#pragma unroll
      for (int u = 0; u < QV; ++u) acc = lz_fmac(v[u], v[u], acc);
      const C n2 = colk::warp_allsum(lz_fin(acc));
      if (fp32_hi(n2) > 0.25f) {
        const C inv = rcp_(sqrt_(n2));
#pragma unroll
        for (int u = 0; u < QV; ++u) {
          const int i = lane + 32 * u;
          if (i < m) Vout[i + (size_t)p * ldV] = mul(v[u], inv);
        }
        __syncwarp();
        ++cand;
        break;
      }
    }
  }
}

// ---- thick-bounds recovery (Alg. 3 line 4) ------------------------------------------
// T_new (ab x rho) = T_old (ab x r) * S0 (r x rho), column-major FP64: the recovered first
// core S0 absorbed into the core to its left
__global__ void k_merge_core(const double* __restrict__ Told, const double* __restrict__ S0,
                             int ab, int r, int rho, double* __restrict__ Tnew) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)ab * rho;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % ab), c = (int)(idx / ab);
    double acc = 0.0;
    for (int t = 0; t < r; ++t) acc = fma(Told[i + (int64_t)t * ab], S0[t + (int64_t)c * r], acc);
    Tnew[idx] = acc;
  }
}

// ranks of the thick train: r_0..r_{p-1} of the reduced train, then rho_1..rho_{q+1} of the
// recovery; err2 = the two discarded energies
__global__ void k_join_ranks(const int64_t* r1, int p, const int64_t* r2, int q, int64_t* out,
                             const double* e12, double* err2_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (out) {
    for (int i = 0; i < p; ++i) out[i] = r1[i];
    for (int i = 1; i <= q + 1; ++i) out[p + i - 1] = r2[i];
  }
  if (err2_out) *err2_out = e12[0] + e12[1];
}

// ---- rank choice: Alg. 2 lines 7-8 --------------------------------------------
__global__ void k_truncate(const double* __restrict__ sigma, int64_t rows, int step_i, int n_next,
                           int r_max, double tol2_over_dm1, DevState* st,
                           double* __restrict__ sigma_out, int64_t* __restrict__ ranks_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = st->m[step_i];
  const int s = (int)((int64_t)m < rows ? m : rows);
  double total = 0.0;
  for (int k = s - 1; k >= 0; --k) total += sigma[k] * sigma[k];
  if (!st->first_done) {
    st->delta2 = tol2_over_dm1 * total;  // delta^2 = eps^2/(d-1) ||Sigma_first||_F^2
    st->first_done = 1;
  }
  const double d2 = st->delta2;
  int r_delta = s;
  if (d2 > 0.0) {
    // smallest j with sigma_{j+1}^2 + ... <= delta^2 (tail summed from the smallest value)
    double tail = 0.0;
    r_delta = s;
    for (int j = s - 1; j >= 0; --j) {
      const double nt = tail + sigma[j] * sigma[j];
      if (nt <= d2) { r_delta = j; tail = nt; } else break;
    }
  }
  int r = r_max;
  if (r_delta < r) r = r_delta;
  if (s < r) r = s;
  if (r < 1) r = 1;
  double disc = 0.0;
  for (int k = s - 1; k >= r; --k) disc += sigma[k] * sigma[k];
  st->err2 += disc;
  st->r[step_i - 1] = r;
  st->m[step_i - 1] = n_next * r;
  // sigma of X itself: the unfoldings were read as X 2^-k (exact power of two)
  if (sigma_out) for (int k = 0; k < s; ++k) sigma_out[k] = ldexp(sigma[k], st->xr.k);
  if (ranks_out) ranks_out[step_i - 1] = r;
}

template <class C>
__global__ void k_core(const C* __restrict__ V, int ldV, const DevState* st, int step_i,
                       double* __restrict__ core) {
  const int m = st->m[step_i];
  const int r = st->r[step_i - 1];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)r * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % r);
    const int j = (int)(idx / r);
    core[idx] = to_f64(V[j + (size_t)a * ldV]);  // T[a + r j] = V[j][a]
  }
}

__global__ void k_set_rank(DevState* st, int step_i, int n_next, int r) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->r[step_i - 1] = r;
  st->m[step_i - 1] = n_next * r;
}

// dst = src as FP64, times 2^xr->k when xr is given (a result of an input read as X 2^-k)
template <class S>
__global__ void k_copy_mat_f64(const S* __restrict__ src, int64_t lds, int rows, int cols,
                               int upper, double* __restrict__ dst, int64_t ldd, const XRange* xr) {
  const int k2 = xr ? xr->k : 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % rows), k = (int)(idx / rows);
    double v = ldexp(to_f64(ld_as<df>(src[i + k * lds])), k2);
    if (upper && i > k) v = 0.0;
    dst[i + k * ldd] = v;
  }
}
template <>
__global__ void k_copy_mat_f64<double>(const double* __restrict__ src, int64_t lds, int rows,
                                       int cols, int upper, double* __restrict__ dst, int64_t ldd,
                                       const XRange* xr) {
  const int k2 = xr ? xr->k : 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % rows), k = (int)(idx / rows);
    double v = ldexp(src[i + k * lds], k2);
    if (upper && i > k) v = 0.0;
    dst[i + k * ldd] = v;
  }
}

__global__ void k_core_identity(int m, double* core) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)m * m;
       idx += (int64_t)gridDim.x * blockDim.x)
    core[idx] = (idx % m == idx / m) ? 1.0 : 0.0;
}

template <class S>
__global__ void k_to_f64(const S* __restrict__ src, int64_t count, double* __restrict__ dst,
                         const XRange* xr) {
  const int k2 = xr ? xr->k : 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[idx] = ldexp(to_f64(ld_as<df>(src[idx])), k2);
}
template <>
__global__ void k_to_f64<double>(const double* __restrict__ src, int64_t count, double* __restrict__ dst,
                                 const XRange* xr) {
  const int k2 = xr ? xr->k : 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[idx] = ldexp(src[idx], k2);
}

// largest encoded exponent of a strided sample of X (at most 64 Ki entries, spread over
// the whole tensor so that column and block scales are seen): one atomic per warp
template <class S>
__global__ void k_range_sample(const S* __restrict__ X, int64_t count, int64_t nsample,
                               XRange* xr) {
  int e = 0;
  const int64_t stride = count / nsample;  // >= 1: nsample <= count
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nsample;
       j += (int64_t)gridDim.x * blockDim.x)
    e = max(e, expo_enc(X[j * stride]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0 && e) atomicMax(&xr->sample, e);
}

// after the first pass of the first TSQR level: keep its shift, or run it again with the
// shift of the largest magnitude it met
__global__ void k_range_decide(XRange* xr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k_try = xr_shift_for(xr->sample);
  const bool redo = xr_needs_redo(k_try, xr->seen);
  xr->redo = redo ? 1 : 0;
  xr->k = redo ? xr_shift_for(xr->seen) : k_try;
}

__global__ void k_fill_nan(double* dst, int64_t count) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[idx] = __longlong_as_double(0x7FF8000000000000ll);
}

struct InitArgs {
  int d;
  int n[40];
};

__global__ void k_init_state(DevState* st, InitArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->status = 0;
  st->xr = XRange{0, 0, 0, 0};
  st->first_done = 0;
  st->delta2 = 0.0;
  st->err2 = 0.0;
  for (int i = 0; i < 40; ++i) { st->m[i] = 0; st->r[i] = 1; st->sweeps[i] = 0; }
  st->m[a.d] = a.n[a.d - 1];  // W^(d) has n_d columns (r_d = 1)
}

__global__ void k_finish(const DevState* st, int d, int64_t* ranks_out, double* err2_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ranks_out) {
    ranks_out[0] = 1;
    ranks_out[d] = 1;
    for (int i = 1; i < d; ++i) ranks_out[i] = st->r[i];
  }
  if (err2_out) *err2_out = ldexp(st->err2, 2 * st->xr.k);
}

inline unsigned grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (unsigned)g;
}

}  // namespace

size_t jacobi_scratch_bytes(Fmt comp, int m_max) {
  const int mp = m_max + (m_max & 1);
  return 2ull * mp * mp * fmt_bytes(comp);
}

template <class C, class RI, int G>
static void run_jacobi_g(const void* R, int64_t ldR, const int* m_dev, int m_max, void* Ag,
                         void* Vg, int ldA, int smem_ok, size_t smem, double* sigma, void* Vout,
                         int ldV, int* status, int* sweeps_out, int sweeps, cudaStream_t s) {
  const int mp = m_max + (m_max & 1);
  int threads = ((mp / 2) * G + 31) / 32 * 32;
  if (threads < 64) threads = 64;
  if (threads > 1024) threads = 1024;
  auto k = k_jacobi<C, RI, G>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<1, threads, smem, s>>>(static_cast<const RI*>(R), ldR, m_dev, m_max, static_cast<C*>(Ag),
                             static_cast<C*>(Vg), ldA, smem_ok, sigma, static_cast<C*>(Vout), ldV,
                             status, sweeps_out, sweeps);
}

template <class C, class RI>
static void run_jacobi(const void* R, int64_t ldR, const int* m_dev, int m_max, void* Ag,
                       void* Vg, int ldA, int smem_ok, size_t smem, double* sigma, void* Vout,
                       int ldV, int* status, int* sweeps_out, int sweeps, cudaStream_t s) {
  // lanes per column pair: 16 up to m = 128 (measured on GB300 for m = 16..48 against 8
  // and 32), tunable through "svd.g"
  const int g = tune_get("svd.g", 16);
  if (g == 32 && m_max <= 64)
    run_jacobi_g<C, RI, 32>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (g == 8 && m_max <= 128)
    run_jacobi_g<C, RI, 8>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (m_max <= 128)
    run_jacobi_g<C, RI, 16>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (m_max <= 256)
    run_jacobi_g<C, RI, 16>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else
    run_jacobi_g<C, RI, 32>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
}

cudaError_t launch_jacobi(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                          int m_max, void* Ag, void* Vg, int ldA, double* sigma, void* Vout,
                          int ldV, int* status, int* sweeps_out, cudaStream_t s) {
  // m > 48: spread the columns over a thread-block cluster when one fits; the block-cyclic
  // ordering first, then the ring ordering
  if (m_max > 48 && tune_get("svd.block", 1)) {
    int bnpl = 0;
    const int bnc = jacobi_block_plan(comp, m_max, &bnpl);
    if (bnc > 0) {
      const cudaError_t e = launch_jacobi_block(comp, rin, R, ldR, m_dev, m_max, bnc, bnpl, sigma,
                                                Vout, ldV, status, sweeps_out, s);
      if (e == cudaSuccess) return e;
      cudaGetLastError();  // launch refused (no resident cluster of that size)
    }
  }
  int npl = 0;
  const int nc = tune_get("svd.cluster", 1) ? jacobi_cluster_plan(comp, m_max, &npl) : 0;
  if (nc > 0) {
    for (int cand : {nc, nc == 16 ? 8 : 16}) {
      const int np = cand == nc ? npl : jacobi_cluster_npl(comp, m_max, cand);
      if (!np) continue;
      const cudaError_t e = launch_jacobi_cluster(comp, rin, R, ldR, m_dev, m_max, cand, np, sigma,
                                                  Vout, ldV, status, sweeps_out, Vg, ldA, s);
      if (e == cudaSuccess) return e;
      cudaGetLastError();  // launch refused (no resident cluster of that size)
    }
  }
  const int mp = m_max + (m_max & 1);
  const size_t need = 2ull * ldA * mp * fmt_bytes(comp);
  const int smem_ok = need <= 200 * 1024 ? 1 : 0;
  const size_t smem = (smem_ok ? need : 0) + (size_t)mp * fmt_bytes(comp);
  const int sweeps = 60;
  if (comp == Fmt::DF && rin == Fmt::DF)
    run_jacobi<df, df>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (comp == Fmt::DF && rin == Fmt::F64)
    run_jacobi<df, double>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (comp == Fmt::DF && rin == Fmt::F32)
    run_jacobi<df, float>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else if (comp == Fmt::F64 && rin == Fmt::F64)
    run_jacobi<double, double>(R, ldR, m_dev, m_max, Ag, Vg, ldA, smem_ok, smem, sigma, Vout, ldV, status, sweeps_out, sweeps, s);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

bool jacobi_wide_fits(Fmt comp, int rows, int m_max) {
  return rows >= 1 && rows < m_max && m_max <= kMaxM && (comp == Fmt::DF || comp == Fmt::F64);
}
// global scratch the wide kernel needs for its working copy (0: it fits in shared memory)
size_t jacobi_wide_gbytes(Fmt comp, int rows, int m_max) {
  const size_t es = fmt_bytes(comp);
  const int ncp = rows + (rows & 1);
  const size_t need = (size_t)ncp * m_max * es + (size_t)ncp * (es + sizeof(int));
  return need <= max_smem_optin() - 4096 ? 0 : (size_t)ncp * m_max * es;
}

template <class C, class WI, int G>
static cudaError_t run_wide_g(const void* W, int64_t ldW, int rows, const int* m_dev, int m_max,
                              double* sigma, void* Vout, int ldV, int* status, int* sweeps_out,
                              void* gscr, cudaStream_t s) {
  const int ncp = rows + (rows & 1);
  const size_t es = sizeof(C);
  const bool glob = gscr != nullptr;
  const size_t smem = (glob ? 0 : (size_t)ncp * m_max * es) + (size_t)ncp * (es + sizeof(int));
  int threads = ((ncp / 2) * G + 31) / 32 * 32;
  if (threads < 64) threads = 64;
  if (threads > 1024) threads = 1024;
  auto k = k_jacobi_wide<C, WI, G>;
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<1, threads, smem, s>>>(static_cast<const WI*>(W), ldW, rows, m_dev, m_max, m_max, sigma,
                             static_cast<C*>(Vout), ldV, status, sweeps_out, 60,
                             static_cast<C*>(gscr));
  return cudaGetLastError();
}

template <class C, class WI>
static cudaError_t run_wide(const void* W, int64_t ldW, int rows, const int* m_dev, int m_max,
                            double* sigma, void* Vout, int ldV, int* status, int* sweeps_out,
                            void* gscr, cudaStream_t s) {
  // lanes per column pair: about 8-16 elements of a column per lane
  const int g = tune_get("svd.wide_g", m_max >= 256 ? 32 : m_max >= 64 ? 16 : 8);
  if (g == 32) return run_wide_g<C, WI, 32>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, gscr, s);
  if (g == 16) return run_wide_g<C, WI, 16>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, gscr, s);
  return run_wide_g<C, WI, 8>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, gscr, s);
}

cudaError_t launch_jacobi_wide(Fmt comp, Fmt win, const void* W, int64_t ldW, int rows,
                               const int* m_dev, int m_max, double* sigma, void* Vout, int ldV,
                               int* status, int* sweeps_out, void* gscr, cudaStream_t s) {
  if (!jacobi_wide_fits(comp, rows, m_max)) return cudaErrorInvalidValue;
  // the working copy in shared memory when it fits, else in gscr (jacobi_wide_gbytes)
  void* g = jacobi_wide_gbytes(comp, rows, m_max) ? gscr : nullptr;
  if (jacobi_wide_gbytes(comp, rows, m_max) && !gscr) return cudaErrorInvalidValue;
  if (comp == Fmt::DF && win == Fmt::DF)
    return run_wide<df, df>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, g, s);
  if (comp == Fmt::DF && win == Fmt::F64)
    return run_wide<df, double>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, g, s);
  if (comp == Fmt::DF && win == Fmt::F32)
    return run_wide<df, float>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, g, s);
  if (comp == Fmt::F64 && win == Fmt::F64)
    return run_wide<double, double>(W, ldW, rows, m_dev, m_max, sigma, Vout, ldV, status, sweeps_out, g, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_truncate(const double* sigma, int64_t rows, int step_i, int n_next, int r_max,
                            double tol2_over_dm1, DevState* st, double* sigma_out_step,
                            int64_t* ranks_out, cudaStream_t s) {
  k_truncate<<<1, 32, 0, s>>>(sigma, rows, step_i, n_next, r_max, tol2_over_dm1, st,
                              sigma_out_step, ranks_out);
  return cudaGetLastError();
}

cudaError_t launch_core(Fmt vfmt, const void* V, int ldV, const DevState* st, int step_i,
                        double* core, cudaStream_t s) {
  if (vfmt == Fmt::DF)
    k_core<df><<<64, 256, 0, s>>>((const df*)V, ldV, st, step_i, core);
  else if (vfmt == Fmt::F64)
    k_core<double><<<64, 256, 0, s>>>((const double*)V, ldV, st, step_i, core);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_set_rank(DevState* st, int step_i, int n_next, int r, cudaStream_t s) {
  k_set_rank<<<1, 32, 0, s>>>(st, step_i, n_next, r);
  return cudaGetLastError();
}

cudaError_t launch_copy_mat_f64(Fmt f, const void* src, int64_t lds, int rows, int cols, int upper,
                                double* dst, int64_t ldd, cudaStream_t s, const XRange* xr) {
  const unsigned g = grid_for((int64_t)rows * cols, 256);
  if (f == Fmt::F64) k_copy_mat_f64<double><<<g, 256, 0, s>>>((const double*)src, lds, rows, cols, upper, dst, ldd, xr);
  else if (f == Fmt::DF) k_copy_mat_f64<df><<<g, 256, 0, s>>>((const df*)src, lds, rows, cols, upper, dst, ldd, xr);
  else k_copy_mat_f64<float><<<g, 256, 0, s>>>((const float*)src, lds, rows, cols, upper, dst, ldd, xr);
  return cudaGetLastError();
}

cudaError_t launch_core_identity(int m, double* core, cudaStream_t s) {
  k_core_identity<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(m, core);
  return cudaGetLastError();
}

cudaError_t launch_merge_core(const double* Told, const double* S0, int ab, int r, int rho,
                              double* Tnew, cudaStream_t s) {
  const int64_t n = (int64_t)ab * rho;
  k_merge_core<<<grid_for(n, 256), 256, 0, s>>>(Told, S0, ab, r, rho, Tnew);
  return cudaGetLastError();
}

cudaError_t launch_join_ranks(const int64_t* r1, int p, const int64_t* r2, int q, int64_t* out,
                              const double* e12, double* err2_out, cudaStream_t s) {
  k_join_ranks<<<1, 32, 0, s>>>(r1, p, r2, q, out, e12, err2_out);
  return cudaGetLastError();
}

cudaError_t launch_convert_to_f64(Fmt f, const void* src, int64_t count, double* dst,
                                  cudaStream_t s, const XRange* xr) {
  if (count <= 0) return cudaSuccess;
  const unsigned g = grid_for(count, 256);
  if (f == Fmt::F64) k_to_f64<double><<<g, 256, 0, s>>>((const double*)src, count, dst, xr);
  else if (f == Fmt::DF) k_to_f64<df><<<g, 256, 0, s>>>((const df*)src, count, dst, xr);
  else k_to_f64<float><<<g, 256, 0, s>>>((const float*)src, count, dst, xr);
  return cudaGetLastError();
}

cudaError_t launch_range_sample(Fmt f, const void* X, int64_t count, XRange* xr, cudaStream_t s) {
  if (f != Fmt::F64 && f != Fmt::F32) return cudaErrorInvalidValue;
  if (count <= 0) return cudaSuccess;
  const int64_t ns = count < 65536 ? count : 65536;
  const unsigned g = grid_for(ns, 256) < 64 ? grid_for(ns, 256) : 64;
  if (f == Fmt::F64)
    k_range_sample<double><<<g, 256, 0, s>>>(static_cast<const double*>(X), count, ns, xr);
  else
    k_range_sample<float><<<g, 256, 0, s>>>(static_cast<const float*>(X), count, ns, xr);
  return cudaGetLastError();
}

__global__ void k_range_set_sample(XRange* xr, int enc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) xr->sample = enc;
}

cudaError_t launch_range_set_sample(XRange* xr, int enc, cudaStream_t s) {
  k_range_set_sample<<<1, 32, 0, s>>>(xr, enc);
  return cudaGetLastError();
}

cudaError_t launch_range_decide(XRange* xr, cudaStream_t s) {
  k_range_decide<<<1, 32, 0, s>>>(xr);
  return cudaGetLastError();
}

cudaError_t launch_fill_nan(double* dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_fill_nan<<<grid_for(count, 256), 256, 0, s>>>(dst, count);
  return cudaGetLastError();
}

cudaError_t launch_init_state(DevState* st, int d, const int64_t* n_host, cudaStream_t s) {
  InitArgs a;
  a.d = d;
  for (int i = 0; i < 40; ++i) a.n[i] = i < d ? (int)n_host[i] : 0;
  k_init_state<<<1, 32, 0, s>>>(st, a);
  return cudaGetLastError();
}

cudaError_t launch_finish(const DevState* st, int d, int64_t* ranks_out, double* err2_out,
                          cudaStream_t s) {
  k_finish<<<1, 32, 0, s>>>(st, d, ranks_out, err2_out);
  return cudaGetLastError();
}

// ---- tt_small_svd_noalloc: the Jacobi SVD with its scratch in a static array -----
//
// For callers that cannot allocate device memory (see include/tt_svd.h).  The
// scratch lives in this file-scope device array, so the entry point below
// calls no cudaMalloc/cudaFree.  Every GPU that loads the library reserves it
// until the process exits.
namespace {
constexpr int kNoAllocMaxM = 256;
constexpr size_t kNoAllocDf = (size_t)kNoAllocMaxM * kNoAllocMaxM;  // elements of one m x m df matrix
// layout: [0, 256) status word | A | V (Jacobi working copies) | V result (float-float)
constexpr size_t kNoAllocBytes = 256 + 3 * kNoAllocDf * sizeof(df);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

// the device address of g_noalloc_scratch on the current device; looked up once per
// device (cudaGetSymbolAddress with that device current), then cached
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// a sweep limit or a non-finite value (a status bit, or a sigma that is not finite):
// report it as sigma[0] = NaN
__global__ void k_noalloc_mark(const int* status, double* sigma, int m) {
  bool bad = *status != 0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) bad |= !isfinite(sigma[k]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) sigma[0] = __longlong_as_double(0x7FF8000000000000ll);
}
}  // namespace

}  // namespace tt

extern "C" tt_status tt_small_svd_noalloc(const double* R, int m, double* sigma, double* V,
                                         void* stream) {
  using namespace tt;
  if (!R || !sigma || !V) return TT_EINVAL;
  if (m < 1 || m > kNoAllocMaxM) {
    set_last_error_text("tt_small_svd_noalloc: m must be in [1, 256] (size of its static scratch)");
    return TT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) {
    char buf[192];
    snprintf(buf, sizeof(buf), "tt_small_svd_noalloc: scratch address lookup: %s", cudaGetErrorString(e));
    set_last_error_text(buf);
    return TT_ECUDA;
  }
  const int mp = m + (m & 1);
  char* b = static_cast<char*>(base);
  int* status = reinterpret_cast<int*>(b);
  df* A = reinterpret_cast<df*>(b + 256);
  df* Vw = A + kNoAllocDf;
  df* Vres = Vw + kNoAllocDf;
  // the status word keeps the previous call's value: clear it; A, V and the result are
  // written in full by the kernels before they are read
  auto fail = [](const char* what, cudaError_t err) {
    char buf[192];
    snprintf(buf, sizeof(buf), "tt_small_svd_noalloc: %s: %s", what, cudaGetErrorString(err));
    set_last_error_text(buf);
    return TT_ECUDA;
  };
  if ((e = cudaMemsetAsync(status, 0, sizeof(int), s)) != cudaSuccess)
    return fail("clearing the status word", e);
  if ((e = launch_jacobi(Fmt::DF, Fmt::F64, R, m, nullptr, m, A, Vw, mp, sigma, Vres, mp, status,
                         nullptr, s)) != cudaSuccess)
    return fail("Jacobi launch", e);
  if ((e = launch_copy_mat_f64(Fmt::DF, Vres, mp, m, m, 0, V, m, s)) != cudaSuccess)
    return fail("copy of V", e);
  k_noalloc_mark<<<1, 256, 0, s>>>(status, sigma, m);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("status mark launch", e);
  return TT_OK;
}
