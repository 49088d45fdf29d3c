// tsmm.cu -- Y = W V(:, 0:r) (Alg. 2 line 11; TSMM of Sec. 4.1.2) and the
// uniform[0,1) Philox4x32-10 input generator.
//
// W is rows x m column-major.  With the unpadded layouts used here the
// reshape of line 11 is a view: the rows x r product, column-major with
// leading dimension rows, is already W^(i-1) = rows/n_{i-1} x (n_{i-1} r).
// A CTA stages a tile of `tr` rows x m of W in shared memory (row-major, odd
// stride) with coalesced loads along the rows, V(:, 0:r) once per CTA, and
// computes the tr x r outputs with consecutive threads on consecutive rows
// (coalesced stores).
#include <algorithm>

#include "tsqr_kernels.cuh"

namespace tt {

namespace {

template <class C, class S, class VS, class SO>
__global__ void __launch_bounds__(256)
k_tsmm(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
       int m_val, const VS* __restrict__ V, int ldV, const int* __restrict__ r_ptr, int r_val,
       SO* __restrict__ Y, int64_t ldy, int tr, int mstr, int m_max, int r_max, int rc,
       int* status, const XRange* xr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XRead<C, S> rd;
  rd.set(xr ? xr->k : 0, xr != nullptr);
  const int m = m_ptr ? *m_ptr : m_val;
  const int r = r_ptr ? *r_ptr : r_val;
  if (m < 1 || m > m_max || r < 1 || r > r_max || r > m || rc < 1) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  C* Vs = reinterpret_cast<C*>(smem_raw);            // chunk of V: Vs[k * rc + (c - c0)]
  C* T = Vs + (size_t)m_max * rc;                    // tile of W: T[i * mstr + k]
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool v_once = rc >= r;                       // all of V(:, 0:r) fits: load it once
  if (v_once)
    for (int idx = tid; idx < m * r; idx += nt) {
      const int k = idx / r, c = idx % r;
      Vs[k * rc + c] = ld_as<C>(V[k + (size_t)c * ldV]);
    }
  const int64_t ntiles = (rows + tr - 1) / tr;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * tr;
    __syncthreads();
    for (int idx = tid; idx < tr * m; idx += nt) {
      const int i = idx % tr, k = idx / tr;
      const int64_t row = r0 + i;
      T[(size_t)i * mstr + k] = row < rows ? rd(W[row + (int64_t)k * ld]) : Tr<C>::zero();
    }
    for (int c0 = 0; c0 < r; c0 += rc) {
      const int cn = (r - c0) < rc ? (r - c0) : rc;
      __syncthreads();
      if (!v_once)
        for (int idx = tid; idx < m * cn; idx += nt) {
          const int k = idx / cn, c = idx % cn;
          Vs[k * rc + c] = ld_as<C>(V[k + (size_t)(c0 + c) * ldV]);
        }
      __syncthreads();
      for (int idx = tid; idx < tr * cn; idx += nt) {
        const int i = idx % tr, c = idx / tr;
        const int64_t row = r0 + i;
        const C* ti = T + (size_t)i * mstr;
        C acc = Tr<C>::zero();
        for (int k = 0; k < m; ++k) acc = fmac(ti[k], Vs[k * rc + c], acc);
        if (row < rows) Y[row + (int64_t)(c0 + c) * ldy] = st_as<SO>(acc);
      }
    }
  }
}

// Register-blocked form: V(:, 0:r) sits in shared memory (zero-padded to a multiple of
// CPT columns); thread t owns rows base + t + 256 q (q < RPT) and CPT output columns at
// a time, streaming its rows of W from global memory once per column chunk (coalesced
// across the threads) and accumulating RPT x CPT products in registers.
template <int RPT, int CPT, int MINB, class C, class S, class VS, class SO>
__global__ void __launch_bounds__(256, MINB)
k_tsmm_rb(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
          int m_val, const VS* __restrict__ V, int ldV, const int* __restrict__ r_ptr, int r_val,
          SO* __restrict__ Y, int64_t ldy, int m_max, int r_max, int* status,
          const XRange* xr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XRead<C, S> rd;
  rd.set(xr ? xr->k : 0, xr != nullptr);
  const int m = m_ptr ? *m_ptr : m_val;
  const int r = r_ptr ? *r_ptr : r_val;
  if (m < 1 || m > m_max || r < 1 || r > r_max || r > m) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int rp = (r + CPT - 1) / CPT * CPT;
  C* Vs = reinterpret_cast<C*>(smem_raw);  // Vs[k * rp + c]
  for (int idx = threadIdx.x; idx < m * rp; idx += blockDim.x) {
    const int k = idx / rp, c = idx % rp;
    Vs[idx] = c < r ? ld_as<C>(V[k + (size_t)c * ldV]) : Tr<C>::zero();
  }
  __syncthreads();
  const int64_t step = (int64_t)gridDim.x * 256 * RPT;
  for (int64_t base = (int64_t)blockIdx.x * 256 * RPT; base < rows; base += step) {
    int64_t row[RPT];
    bool ok[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      row[q] = base + threadIdx.x + 256 * q;
      ok[q] = row[q] < rows;
    }
    for (int c0 = 0; c0 < r; c0 += CPT) {
      // lazy float-float accumulators (normalised once, at the store)
      decltype(lz(Tr<C>::zero())) acc[RPT][CPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) acc[q][cc] = lz(Tr<C>::zero());
#pragma unroll 8
      for (int k = 0; k < m; ++k) {
        C w[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          w[q] = ok[q] ? rd(W[row[q] + (int64_t)k * ld]) : Tr<C>::zero();
        const C* vk = Vs + k * rp + c0;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const C v = vk[cc];
#pragma unroll
          for (int q = 0; q < RPT; ++q) acc[q][cc] = lz_fmac(w[q], v, acc[q][cc]);
        }
      }
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc)
        if (c0 + cc < r)
#pragma unroll
          for (int q = 0; q < RPT; ++q)
            if (ok[q]) Y[row[q] + (int64_t)(c0 + cc) * ldy] = st_as<SO>(lz_fin(acc[q][cc]));
    }
  }
}

template <Fmt F> using T_ = typename FT<F>::T;

template <int RPT, int CPT, int MINB, class C, class S, class VS, class SO>
cudaError_t run_rb(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                   const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                   cudaStream_t s) {
  auto k = k_tsmm_rb<RPT, CPT, MINB, C, S, VS, SO>;
  if (c.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)c.ctas, 256, c.smem, s>>>(static_cast<const S*>(W), rows, ld, m_dev, c.m_max,
                                          static_cast<const VS*>(V), ldV, r_dev, c.r_max,
                                          static_cast<SO*>(Y), ldy, c.m_max, c.r_max, status,
                                          c.xr);
  return cudaGetLastError();
}

template <class C, class S, class VS, class SO>
cudaError_t run(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                cudaStream_t s) {
  if (c.kind == 1) {
    // one row per thread and several CTAs per SM keep many loads in flight
    switch (c.cpt) {
      case 1: return run_rb<1, 1, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 2: return run_rb<1, 2, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 4: return run_rb<1, 4, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 5: return run_rb<1, 5, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 8: return run_rb<1, 8, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 10: return run_rb<1, 10, 4, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 16: return run_rb<1, 16, 2, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 20: return run_rb<1, 20, 2, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      case 25: return run_rb<1, 25, 2, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
      default: return run_rb<1, 32, 2, C, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
    }
  }
  auto k = k_tsmm<C, S, VS, SO>;
  if (c.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)c.ctas, 256, c.smem, s>>>(static_cast<const S*>(W), rows, ld, m_dev, c.m_max,
                                          static_cast<const VS*>(V), ldV, r_dev, c.r_max,
                                          static_cast<SO*>(Y), ldy, c.tr, c.mstr, c.m_max,
                                          c.r_max, c.rc, status, c.xr);
  return cudaGetLastError();
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------------
__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}
__device__ __forceinline__ double words_to_unit(uint32_t x, uint32_t y) {
  return ((double)(x >> 5) * 67108864.0 + (double)(y >> 6)) * (1.0 / 9007199254740992.0);
}

template <class T>
__global__ void k_gen(T* __restrict__ out, int64_t count, uint64_t seed, int64_t start) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int64_t b0 = start / 2, b1 = (start + count - 1) / 2;
  for (int64_t b = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= b1;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c0 = (uint32_t)b, c1 = (uint32_t)((uint64_t)b >> 32), c2 = 0, c3 = 0;
    philox10(c0, c1, c2, c3, k0, k1);
    const int64_t e0 = 2 * b - start;
    if (e0 >= 0 && e0 < count) out[e0] = (T)words_to_unit(c0, c1);
    if (e0 + 1 >= 0 && e0 + 1 < count) out[e0 + 1] = (T)words_to_unit(c2, c3);
  }
}

}  // namespace

TsmmCfg plan_tsmm(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max, int64_t rows,
                  int nsm) {
  TsmmCfg c;
  c.in = in; c.comp = comp; c.vfmt = vfmt; c.out = out;
  c.m_max = m_max; c.r_max = r_max;
  c.mstr = m_max | 1;
  const size_t es = fmt_bytes(comp);
  const size_t budget = 200 * 1024;
  // float-float: the tensor-core form (Ozaki splitting) where its exact sums hold
  if (tsmm_tc_ok(in, comp, vfmt, out, m_max, r_max)) {
    c.kind = 3;
    c.cpt = 0;
    c.tr = 128;
    c.rc = 1;
    c.smem = tsmm_tc_smem(m_max, r_max);
    const int64_t ntiles = (rows + 127) / 128;
    c.ctas = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nsm));
    return c;
  }
  if (tsmm_oz_ok(in, comp, vfmt, out, m_max, r_max)) {
    c.kind = 2;
    c.cpt = 0;
    c.tr = 64;
    // tile buffers per CTA: two (the next tile's copy overlaps this tile) or one
    // (more CTAs per SM overlap each other's copies)
    c.rc = tune_get("tsmm.oz_nbuf", 1) == 2 ? 2 : 1;
    c.smem = tsmm_oz_smem(m_max, r_max, c.rc, comp == Fmt::F64);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (c.smem + 1024)));
    const int64_t ntiles = (rows + 63) / 64;
    c.ctas = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nsm * per_sm));
    // the native FP64 form: the tcgen05 pipeline where it applies, this launch as its
    // fallback (a W whose tensor map cannot be made)
    if (tsmm_ws_ok(in, comp, vfmt, out, m_max, r_max) && rows >= 128) {
      c.fb_rc = c.rc;
      c.fb_smem = c.smem;
      c.fb_ctas = c.ctas;
      c.kind = 4;
      c.tr = 128;
      c.smem = tsmm_ws_smem(m_max);
      c.ctas = std::max<int64_t>(1, std::min<int64_t>((rows + 127) / 128, (int64_t)nsm));
    }
    return c;
  }
  // register-blocked form when V(:, 0:r) fits in shared memory
  // output columns per pass: the smallest instantiated width >= r_max (r_max = 50 runs as 2 x 25)
  static const int widths[] = {1, 2, 4, 5, 8, 10, 16, 20, 25, 32};
  c.cpt = 32;
  for (int w : widths)
    if (w >= r_max) { c.cpt = w; break; }
  if (r_max > 32 && r_max <= 50) c.cpt = 25;
  const int rp = (r_max + c.cpt - 1) / c.cpt * c.cpt;
  if ((size_t)m_max * rp * es <= budget) {
    c.kind = 1;
    c.tr = 0;
    c.rc = 0;
    c.smem = (size_t)m_max * rp * es;
    const int64_t blocks = (rows + 255) / 256;
    const int per_sm = std::min(c.cpt <= 10 ? 4 : 2, c.smem > 100 * 1024 ? 1 : (c.smem > 56 * 1024 ? 2 : 4));
    c.ctas = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)nsm * per_sm));
    return c;
  }
  c.kind = 0;
  // row tile first (at least 32 rows), then as many V columns as still fit
  int tr = 128;
  while (tr > 32 && (size_t)tr * c.mstr * es + (size_t)m_max * es > budget) tr /= 2;
  int rc = r_max;
  while (rc > 1 && (size_t)m_max * rc * es + (size_t)tr * c.mstr * es > budget) rc = (rc + 1) / 2;
  c.tr = tr;
  c.rc = rc;
  c.smem = (size_t)m_max * rc * es + (size_t)tr * c.mstr * es;
  const int64_t ntiles = (rows + tr - 1) / tr;
  const int per_sm = c.smem > 100 * 1024 ? 1 : (c.smem > 56 * 1024 ? 2 : 4);
  int64_t ctas = (int64_t)nsm * per_sm;
  if (ctas > ntiles) ctas = ntiles;
  if (ctas < 1) ctas = 1;
  c.ctas = ctas;
  return c;
}

cudaError_t launch_tsmm(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                        const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                        int64_t ldy, int* status, cudaStream_t s) {
  if (c.kind == 3) return launch_tsmm_tc(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.kind == 2) return launch_tsmm_oz(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.kind == 4) {
    bool used = false;
    const cudaError_t e = launch_tsmm_ws(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s, &used);
    if (used || e != cudaSuccess) return e;
    TsmmCfg o = c;
    o.kind = 2;
    o.tr = 64;
    o.rc = c.fb_rc;
    o.smem = c.fb_smem;
    o.ctas = c.fb_ctas;
    return launch_tsmm_oz(o, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  }
#define TT_TSMM(IN, CO, VF, OUT)                                                                \
  if (c.in == Fmt::IN && c.comp == Fmt::CO && c.vfmt == Fmt::VF && c.out == Fmt::OUT)           \
    return run<T_<Fmt::CO>, T_<Fmt::IN>, T_<Fmt::VF>, T_<Fmt::OUT>>(c, W, rows, ld, m_dev, V, ldV, \
                                                                    r_dev, Y, ldy, status, s);
  TT_TSMM(F64, DF, DF, DF)
  TT_TSMM(DF, DF, DF, DF)
  TT_TSMM(F64, F64, F64, F64)
  TT_TSMM(F32, F32, DF, F32)
  TT_TSMM(F64, DF, F64, F64)
  TT_TSMM(F32, F32, F64, F64)
#undef TT_TSMM
  return cudaErrorInvalidValue;
}

cudaError_t launch_gen_uniform(void* out, Fmt f, int64_t count, uint64_t seed, int64_t start,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks_needed = ((start + count - 1) / 2 - start / 2 + 1 + 255) / 256;
  const unsigned g = (unsigned)(blocks_needed < 152 * 16 ? (blocks_needed < 1 ? 1 : blocks_needed) : 152 * 16);
  if (f == Fmt::F64) k_gen<double><<<g, 256, 0, s>>>((double*)out, count, seed, start);
  else if (f == Fmt::F32) k_gen<float><<<g, 256, 0, s>>>((float*)out, count, seed, start);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace tt
