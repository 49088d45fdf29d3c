// svd_cluster.cu -- one-sided Jacobi SVD of R spread over a thread-block cluster.
//
// Same method as k_jacobi in svd.cu (Hestenes rotations of the columns of
// A = R, V accumulated, round-robin pair ordering), with the columns of A and V
// distributed over the shared memory of NC CTAs of one cluster.
//
// Ordering: the MP columns (m padded with zero columns to a multiple of 2 NC)
// sit in P = MP/2 pair positions, each with a "top" and a "bottom" column; pair
// position s is held by CTA s / npl (npl = P / NC positions per CTA).  After a
// round every column moves one position along the ring of the circle method:
//   top(0) stays, top(1) <- bottom(0), top(s) <- top(s-1) (s >= 2),
//   bottom(s) <- bottom(s+1) (s <= P-2), bottom(P-1) <- top(P-1),
// so that 2P-1 rounds pair every two columns exactly once.  Inside a CTA the
// move is a relabelling of shared-memory slots; only the last top column of a
// CTA (to the next CTA) and its first bottom column (to the previous CTA) cross
// CTAs, written into fixed receive buffers of the neighbour through
// distributed shared memory (one buffer pair per round parity), followed by a
// cluster barrier.  Zero (padding) columns are never rotated.
#include <cooperative_groups.h>
#include <mutex>
#include <type_traits>

#include "tsqr_kernels.cuh"

namespace cg = cooperative_groups;

namespace tt {

namespace {

__device__ __forceinline__ float hi32(df a) { return a.hi; }
__device__ __forceinline__ float hi32(double a) { return (float)a; }
template <class C> __device__ __forceinline__ C pow2s(C a, int e);
template <> __device__ __forceinline__ df pow2s<df>(df a, int e) { return mkdf(ldexpf(a.hi, e), ldexpf(a.lo, e)); }
template <> __device__ __forceinline__ double pow2s<double>(double a, int e) { return ldexp(a, e); }

__device__ __forceinline__ void rotcs(float t, df& c, df& sn) {
  float p, e;
  eft_two_prod(t, t, p, e);
  const df u = add(mkdf(1.f, 0.f), mkdf(p, e));
  df cc = mkdf(rsqrtf(u.hi), 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df r = fnmac(u, mul(cc, cc), mkdf(1.f, 0.f));
    cc = fmac(mul(cc, mkdf(0.5f, 0.f)), r, cc);
  }
  c = cc;
  sn = mul(cc, mkdf(t, 0.f));
}
__device__ __forceinline__ void rotcs(float t, double& c, double& sn) {
  c = 1.0 / sqrt(1.0 + (double)t * (double)t);
  sn = c * (double)t;
}

template <int G>
__device__ __forceinline__ df gsum2(df a, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
    a = add(a, mkdf(__shfl_xor_sync(mask, a.hi, o), __shfl_xor_sync(mask, a.lo, o)));
  return a;
}
template <int G>
__device__ __forceinline__ double gsum2(double a, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(mask, a, o);
  return a;
}

template <class C> __device__ __forceinline__ float ctol(int m);
template <> __device__ __forceinline__ float ctol<df>(int m) { return 2.0e-14f * (float)(m < 8 ? 8 : m); }
template <> __device__ __forceinline__ float ctol<double>(int m) { return 2.5e-16f * (float)(m < 8 ? 8 : m); }

// shared memory per CTA: NSLOT column slots of A (m entries) and V (m entries), with
// NSLOT = 2 npl + 4 (working slots, receive buffers top/bottom x round parity)
template <class C, class RI, int G>
__global__ void __launch_bounds__(512)
k_jacobi_cluster(const RI* __restrict__ R, int64_t ldR, const int* __restrict__ m_ptr, int m_max,
                 int npl, double* __restrict__ sigma, C* __restrict__ Vout, int ldV, int* status,
                 int* sweeps_out, int max_sweeps) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int tslot[64], bslot[64];
  __shared__ int s_rot;
  __shared__ int s_flags[2][16];
  __shared__ float s_red[16];
  __shared__ int s_any;
  const int m = m_ptr ? *m_ptr : m_max;
  const int NC = (int)cl.num_blocks();
  const int c = (int)cl.block_rank();
  const int P = NC * npl;
  const int MP = 2 * P;
  const int nslot = 2 * npl + 4;
  if (m < 1 || m > m_max || MP < m || npl > 64 || npl < 2 || NC > 16) {
    if (threadIdx.x == 0 && c == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;  // uniform over the cluster: every CTA sees the same m, npl and NC
  }
  C* Acol = reinterpret_cast<C*>(smem_raw);              // slot k: Acol[k * m_max + i]
  C* Vcol = Acol + (size_t)nslot * m_max;                // slot k: Vcol[k * m_max + i]
  int* colid = reinterpret_cast<int*>(Vcol + (size_t)nslot * m_max);  // colid[slot]: column id
  double* allnorm = reinterpret_cast<double*>(colid + ((nslot + 1) & ~1));  // allnorm[MP]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nt >> 5;
  const int RT0 = 2 * npl, RB0 = 2 * npl + 2;            // receive buffers (top, bottom) x parity

  // max |R| and ||R||_F^2 (every CTA reads all of R: cheap, and no cross-CTA reduction)
  float mx = 0.f;
  for (int idx = tid; idx < m * m; idx += nt) {
    const int i = idx % m, k = idx / m;
    if (i <= k) mx = fmaxf(mx, fabsf(hi32(ld_as<C>(R[i + (int64_t)k * ldR]))));
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[wid] = mx;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < nwarps; ++w) t = fmaxf(t, s_red[w]);
  int ex = 0;
  if (t > 0.f) frexpf(t, &ex);
  __syncthreads();
  // initial placement: position s = c npl + i holds columns 2s (top) and 2s+1 (bottom)
  if (tid < npl) {
    tslot[tid] = tid;
    bslot[tid] = npl + tid;
  }
  for (int k = 0; k < 2 * npl; ++k) {
    const int s = c * npl + (k < npl ? k : k - npl);
    const int col = 2 * s + (k < npl ? 0 : 1);
    if (tid == 0) colid[k] = col;
    for (int i = tid; i < m; i += nt) {
      C a = Tr<C>::zero();
      if (col < m && i <= col) a = pow2s<C>(ld_as<C>(R[i + (int64_t)col * ldR]), -ex);
      Acol[(size_t)k * m_max + i] = a;
      Vcol[(size_t)k * m_max + i] = (i == col) ? Tr<C>::one() : Tr<C>::zero();
    }
  }
  float fro = 0.f;
  for (int idx = tid; idx < m * m; idx += nt) {
    const int i = idx % m, k = idx / m;
    if (i <= k) {
      const float v = ldexpf(hi32(ld_as<C>(R[i + (int64_t)k * ldR])), -ex);
      fro = fmaf(v, v, fro);
    }
  }
  for (int o = 16; o; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  __syncthreads();
  if (lane == 0) s_red[wid] = fro;
  __syncthreads();
  float frot = 0.f;
  for (int w = 0; w < nwarps; ++w) frot += s_red[w];
  const float tol = ctol<C>(m);
  const float floor_abs = tol * tol * frot;
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  cl.sync();

  // neighbour receive buffers through distributed shared memory
  C* nextA = c + 1 < NC ? cl.map_shared_rank(Acol, c + 1) : nullptr;
  C* nextV = c + 1 < NC ? cl.map_shared_rank(Vcol, c + 1) : nullptr;
  int* nextId = c + 1 < NC ? cl.map_shared_rank(colid, c + 1) : nullptr;
  C* prevA = c > 0 ? cl.map_shared_rank(Acol, c - 1) : nullptr;
  C* prevV = c > 0 ? cl.map_shared_rank(Vcol, c - 1) : nullptr;
  int* prevId = c > 0 ? cl.map_shared_rank(colid, c - 1) : nullptr;
  int* flags0 = cl.map_shared_rank(&s_flags[0][0], 0);

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < MP - 1; ++rnd) {
      const int par = rnd & 1;
      // 1. rotate the local pairs
      for (int i = gid; i < npl; i += ngroups) {
        C* ap = Acol + (size_t)tslot[i] * m_max;
        C* aq = Acol + (size_t)bslot[i] * m_max;
        auto al = lz(Tr<C>::zero()), be = al, ga = al;  // lazy float-float sums
        for (int r = gl; r < m; r += G) {
          const C x = ap[r], y = aq[r];
          al = lz_fmac(x, x, al);
          be = lz_fmac(y, y, be);
          ga = lz_fmac(x, y, ga);
        }
        const C alf = lz_fin(lz_gsum<G>(al, gmask));
        const C bef = lz_fin(lz_gsum<G>(be, gmask));
        const C gaf = lz_fin(lz_gsum<G>(ga, gmask));
        const float gf = fabsf(hi32(gaf));
        const float nf = sqrtf(hi32(alf)) * sqrtf(hi32(bef));
        if (gf > tol * nf && nf > floor_abs && gf > 0.f) {
          const float zf = hi32(sub(bef, alf)) / (2.f * hi32(gaf));
          const float az = fabsf(zf);
          float tf = az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f)));
          if (zf < 0.f) tf = -tf;
          C cs, sn;
          rotcs(tf, cs, sn);
          C* vp = Vcol + (size_t)tslot[i] * m_max;
          C* vq = Vcol + (size_t)bslot[i] * m_max;
          for (int r = gl; r < m; r += G) {
            const C x = ap[r], y = aq[r];
            ap[r] = fnmac(sn, y, mul(cs, x));
            aq[r] = fmac(sn, x, mul(cs, y));
            const C vx = vp[r], vy = vq[r];
            vp[r] = fnmac(sn, vy, mul(cs, vx));
            vq[r] = fmac(sn, vx, mul(cs, vy));
          }
          if (gl == 0) s_rot = 1;
        }
      }
      __syncthreads();
      // 2. send the boundary columns into the neighbours' receive buffers
      if (nextA) {
        const int src = tslot[npl - 1], dst = RT0 + par;
        for (int r = tid; r < m; r += nt) {
          nextA[(size_t)dst * m_max + r] = Acol[(size_t)src * m_max + r];
          nextV[(size_t)dst * m_max + r] = Vcol[(size_t)src * m_max + r];
        }
        if (tid == 0) nextId[dst] = colid[src];
      }
      if (prevA) {
        const int src = bslot[0], dst = RB0 + par;
        for (int r = tid; r < m; r += nt) {
          prevA[(size_t)dst * m_max + r] = Acol[(size_t)src * m_max + r];
          prevV[(size_t)dst * m_max + r] = Vcol[(size_t)src * m_max + r];
        }
        if (tid == 0) prevId[dst] = colid[src];
      }
      cl.sync();
      // 3. move received columns into the freed slots and relabel the slots (positions
      //    are relabelled by one thread each from the old maps; one barrier for both)
      const int oldT = tslot[npl - 1], oldB = bslot[0];
      if (c > 0 && c + 1 < NC) {
        // freed: oldT (sent right), oldB (sent left); received: top from c-1, bottom from c+1
        for (int r = tid; r < m; r += nt) {
          Acol[(size_t)oldT * m_max + r] = Acol[(size_t)(RT0 + par) * m_max + r];
          Vcol[(size_t)oldT * m_max + r] = Vcol[(size_t)(RT0 + par) * m_max + r];
          Acol[(size_t)oldB * m_max + r] = Acol[(size_t)(RB0 + par) * m_max + r];
          Vcol[(size_t)oldB * m_max + r] = Vcol[(size_t)(RB0 + par) * m_max + r];
        }
        if (tid == 0) {
          colid[oldT] = colid[RT0 + par];
          colid[oldB] = colid[RB0 + par];
        }
      } else if (c == 0 && NC > 1) {
        // freed: oldT (sent right); bottom(0) moves to top(1); received: bottom from CTA 1
        for (int r = tid; r < m; r += nt) {
          Acol[(size_t)oldT * m_max + r] = Acol[(size_t)(RB0 + par) * m_max + r];
          Vcol[(size_t)oldT * m_max + r] = Vcol[(size_t)(RB0 + par) * m_max + r];
        }
        if (tid == 0) colid[oldT] = colid[RB0 + par];
      } else if (c + 1 == NC && NC > 1) {
        // freed: oldB (sent left); top(P-1) moves to bottom(P-1); received: top from c-1
        for (int r = tid; r < m; r += nt) {
          Acol[(size_t)oldB * m_max + r] = Acol[(size_t)(RT0 + par) * m_max + r];
          Vcol[(size_t)oldB * m_max + r] = Vcol[(size_t)(RT0 + par) * m_max + r];
        }
        if (tid == 0) colid[oldB] = colid[RT0 + par];
      }
      int ntop = 0, nbot = 0;
      if (tid < npl) {
        const int i = tid;
        const int s = c * npl + i;
        if (s == 0) ntop = tslot[0];
        else if (s == 1) ntop = bslot[0];                 // CTA 0, i = 1 (npl >= 2)
        else if (i >= 1) ntop = tslot[i - 1];
        else ntop = (c + 1 == NC) ? oldB : oldT;          // received top lives in the freed slot
        if (s == P - 1) nbot = tslot[npl - 1];            // last CTA keeps top(P-1) as bottom
        else if (i <= npl - 2) nbot = bslot[i + 1];
        else nbot = (c == 0) ? oldT : oldB;               // received bottom lives in the freed slot
      }
      __syncthreads();  // every old slot index has been read
      if (tid < npl) {
        tslot[tid] = ntop;
        bslot[tid] = nbot;
      }
      __syncthreads();
    }
    // 4. cluster-wide "any rotation in this sweep?"
    const int sp = sweep & 1;
    if (tid == 0) flags0[sp * 16 + c] = s_rot;
    cl.sync();
    if (tid == 0) {
      int any = 0;
      for (int k = 0; k < NC; ++k) any |= flags0[sp * 16 + k];
      s_any = any;
    }
    __syncthreads();
    if (s_any == 0) break;
  }
  if (sweep >= max_sweeps && tid == 0 && c == 0 && status) atomicOr(status, DEV_SVD_NOCONV);
  if (tid == 0 && c == 0 && sweeps_out) *sweeps_out = sweep + 1;

  // 5. norms of every column into every CTA, then rank and write the local columns
  for (int k = wid; k < 2 * npl; k += nwarps) {
    const int slot = k < npl ? tslot[k] : bslot[k - npl];
    C acc = Tr<C>::zero();
    for (int r = lane; r < m; r += 32) acc = fmac(Acol[(size_t)slot * m_max + r], Acol[(size_t)slot * m_max + r], acc);
    acc = gsum2<32>(acc, 0xffffffffu);
    if (lane == 0) {
      const double nv = to_f64(acc);
      const int id = colid[slot];
      for (int q = 0; q < NC; ++q) cl.map_shared_rank(allnorm, q)[id] = nv;
    }
  }
  cl.sync();
  for (int k = tid; k < 2 * npl; k += nt) {
    const int slot = k < npl ? tslot[k] : bslot[k - npl];
    const int id = colid[slot];
    if (id >= m) continue;  // padding column
    const double nk = allnorm[id];
    int rank = 0;
    for (int k2 = 0; k2 < m; ++k2) {
      if (k2 == id) continue;
      const double n2 = allnorm[k2];
      if (n2 > nk || (n2 == nk && k2 < id)) ++rank;
    }
    const double sg = ldexp(sqrt(nk), ex);
    if (!isfinite(sg) && status) atomicOr(status, DEV_NONFINITE);
    sigma[rank] = sg;
    for (int r = 0; r < m; ++r) Vout[r + (size_t)rank * ldV] = Vcol[(size_t)slot * m_max + r];
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

std::mutex g_cl_mu;
int g_cl_ok[2][17];  // [type][NC]: 0 unknown, 1 usable, -1 not usable

}  // namespace

size_t jacobi_cluster_smem(Fmt comp, int m_max, int npl) {
  const int nslot = 2 * npl + 4;
  const int P2 = 2 * 16 * npl;  // allnorm holds up to MP doubles
  return (size_t)2 * nslot * m_max * fmt_bytes(comp) + (size_t)((nslot + 1) & ~1) * 4 +
         (size_t)P2 * sizeof(double) + 16;
}

// positions per CTA for a cluster of nc CTAs and this m (0 if it does not fit)
int jacobi_cluster_npl(Fmt comp, int m_max, int nc) {
  int npl = (m_max + 2 * nc - 1) / (2 * nc);
  if (npl < 2) npl = 2;
  if (npl > 64) return 0;
  return jacobi_cluster_smem(comp, m_max, npl) <= 200 * 1024 ? npl : 0;
}

// preferred cluster size for m (0 = use the single-CTA kernel); the caller falls back
// to the other size if a cluster of the preferred size cannot be resident
int jacobi_cluster_plan(Fmt comp, int m_max, int* npl_out) {
  if (m_max <= 48) return 0;
  const int first = m_max >= 128 ? 16 : 8;
  for (int nc : {first, first == 16 ? 8 : 16}) {
    const int npl = jacobi_cluster_npl(comp, m_max, nc);
    if (npl) {
      *npl_out = npl;
      return nc;
    }
  }
  return 0;
}

template <class C, class RI, int G>
static cudaError_t launch_cl(const void* R, int64_t ldR, const int* m_dev, int m_max, int nc,
                             int npl, double* sigma, void* Vout, int ldV, int* status,
                             int* sweeps_out, cudaStream_t s) {
  auto k = k_jacobi_cluster<C, RI, G>;
  const size_t smem = jacobi_cluster_smem(std::is_same<C, df>::value ? Fmt::DF : Fmt::F64, m_max, npl);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nc > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  int threads = ((npl * G + 31) / 32) * 32;
  if (threads < 128) threads = 128;
  if (threads > 512) threads = 512;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // can a cluster of this size and shared memory be resident at all? (checked once)
  {
    std::lock_guard<std::mutex> lk(g_cl_mu);
    int& ok = g_cl_ok[std::is_same<C, df>::value ? 0 : 1][nc];
    if (ok == 0) {
      int nclusters = 0;
      ok = (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0) ? 1 : -1;
      cudaGetLastError();
    }
    if (ok < 0) return cudaErrorNotSupported;
  }
  return cudaLaunchKernelEx(&cfg, k, static_cast<const RI*>(R), ldR, m_dev, m_max, npl, sigma,
                            static_cast<C*>(Vout), ldV, status, sweeps_out, 60);
}

cudaError_t launch_jacobi_cluster(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                                  int m_max, int nc, int npl, double* sigma, void* Vout, int ldV,
                                  int* status, int* sweeps_out, cudaStream_t s) {
  const bool wide = m_max > 128;
  if (comp == Fmt::DF && rin == Fmt::DF)
    return wide ? launch_cl<df, df, 32>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s)
                : launch_cl<df, df, 16>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s);
  if (comp == Fmt::DF && rin == Fmt::F32)
    return wide ? launch_cl<df, float, 32>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s)
                : launch_cl<df, float, 16>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s);
  if (comp == Fmt::DF && rin == Fmt::F64)
    return wide ? launch_cl<df, double, 32>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s)
                : launch_cl<df, double, 16>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s);
  if (comp == Fmt::F64 && rin == Fmt::F64)
    return wide ? launch_cl<double, double, 32>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s)
                : launch_cl<double, double, 16>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status, sweeps_out, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
