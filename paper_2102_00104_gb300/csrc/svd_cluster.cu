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
// NSLOT = 2 npl + 4 (working slots, receive buffers top/bottom x round parity).  VG: V stays
// in global memory (Vg, column = the logical column id), for m where A and V together do not
// fit: a column of V is only ever touched by the CTA holding the matching column of A, and
// moves between CTAs are ordered by the cluster barriers, so only A's columns travel.
template <class C, class RI, int G, bool VG>
__global__ void __launch_bounds__(512)
k_jacobi_cluster(const RI* __restrict__ R, int64_t ldR, const int* __restrict__ m_ptr, int m_max,
                 int npl, double* __restrict__ sigma, C* __restrict__ Vout, int ldV, int* status,
                 int* sweeps_out, int max_sweeps, C* __restrict__ Vg, int ldVg) {
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
  C* Vcol = Acol + (size_t)nslot * m_max;                // slot k: Vcol[k * m_max + i] (!VG)
  int* colid = reinterpret_cast<int*>(VG ? Vcol : Vcol + (size_t)nslot * m_max);  // column id
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
      if (col < m && i <= col) a = flush_tiny(pow2s<C>(ld_as<C>(R[i + (int64_t)col * ldR]), -ex));
      Acol[(size_t)k * m_max + i] = a;
      if constexpr (VG) {
        if (col < m) Vg[i + (size_t)col * ldVg] = (i == col) ? Tr<C>::one() : Tr<C>::zero();
      } else {
        Vcol[(size_t)k * m_max + i] = (i == col) ? Tr<C>::one() : Tr<C>::zero();
      }
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
  C* nextV = !VG && c + 1 < NC ? cl.map_shared_rank(Vcol, c + 1) : nullptr;
  int* nextId = c + 1 < NC ? cl.map_shared_rank(colid, c + 1) : nullptr;
  C* prevA = c > 0 ? cl.map_shared_rank(Acol, c - 1) : nullptr;
  C* prevV = !VG && c > 0 ? cl.map_shared_rank(Vcol, c - 1) : nullptr;
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
          C* vp = VG ? Vg + (size_t)colid[tslot[i]] * ldVg : Vcol + (size_t)tslot[i] * m_max;
          C* vq = VG ? Vg + (size_t)colid[bslot[i]] * ldVg : Vcol + (size_t)bslot[i] * m_max;
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
          if constexpr (!VG) nextV[(size_t)dst * m_max + r] = Vcol[(size_t)src * m_max + r];
        }
        if (tid == 0) nextId[dst] = colid[src];
      }
      if (prevA) {
        const int src = bslot[0], dst = RB0 + par;
        for (int r = tid; r < m; r += nt) {
          prevA[(size_t)dst * m_max + r] = Acol[(size_t)src * m_max + r];
          if constexpr (!VG) prevV[(size_t)dst * m_max + r] = Vcol[(size_t)src * m_max + r];
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
          Acol[(size_t)oldB * m_max + r] = Acol[(size_t)(RB0 + par) * m_max + r];
          if constexpr (!VG) {
            Vcol[(size_t)oldT * m_max + r] = Vcol[(size_t)(RT0 + par) * m_max + r];
            Vcol[(size_t)oldB * m_max + r] = Vcol[(size_t)(RB0 + par) * m_max + r];
          }
        }
        if (tid == 0) {
          colid[oldT] = colid[RT0 + par];
          colid[oldB] = colid[RB0 + par];
        }
      } else if (c == 0 && NC > 1) {
        // freed: oldT (sent right); bottom(0) moves to top(1); received: bottom from CTA 1
        for (int r = tid; r < m; r += nt) {
          Acol[(size_t)oldT * m_max + r] = Acol[(size_t)(RB0 + par) * m_max + r];
          if constexpr (!VG) Vcol[(size_t)oldT * m_max + r] = Vcol[(size_t)(RB0 + par) * m_max + r];
        }
        if (tid == 0) colid[oldT] = colid[RB0 + par];
      } else if (c + 1 == NC && NC > 1) {
        // freed: oldB (sent left); top(P-1) moves to bottom(P-1); received: top from c-1
        for (int r = tid; r < m; r += nt) {
          Acol[(size_t)oldB * m_max + r] = Acol[(size_t)(RT0 + par) * m_max + r];
          if constexpr (!VG) Vcol[(size_t)oldB * m_max + r] = Vcol[(size_t)(RT0 + par) * m_max + r];
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
    for (int r = 0; r < m; ++r)
      Vout[r + (size_t)rank * ldV] = VG ? Vg[r + (size_t)id * ldVg] : Vcol[(size_t)slot * m_max + r];
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

// sweeps stop early once the largest |cos| rotated in a sweep is below this
constexpr float kEarlyCos = 1e-7f;

// ---- block-cyclic ordering ----------------------------------------------------------------
// The MP = 2 NC npl columns (m padded with zero columns; npl even) form 2 NC blocks of npl
// columns; CTA c holds a top and a bottom block.  A sweep is the circle method on blocks,
// 2 NC - 1 outer rounds: in each, npl cross rounds pair top_i with bottom_{(i+k) mod npl}
// (k = 0..npl-1), and in the first outer round every CTA also pairs the columns inside its
// two blocks (npl - 1 rounds of the circle method inside a block).  Every pair of columns
// meets once per sweep, only __syncthreads separates the inner rounds, and whole blocks
// move between CTAs (distributed shared memory, one cluster barrier) once per outer round.
// Blocks live in four buffers: top = 2p, bottom = 2p + 1 for the parity p of the outer
// round; the moves of an outer round write the other parity's buffers (remote or local).

// rotate the pair (a_p, a_q) (and V's columns) by a group of G lanes; true if rotated
template <class C, int G>
__device__ __forceinline__ bool jacobi_pair(C* ap, C* aq, C* vp, C* vq, int m, int gl,
                                            unsigned gmask, float tol, float floor_abs,
                                            float& maxcos) {
  auto al = lz(Tr<C>::zero()), be = al, ga = al;
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
  if (!(gf > tol * nf && nf > floor_abs && gf > 0.f)) return false;
  maxcos = fmaxf(maxcos, gf / nf);
  const float zf = hi32(sub(bef, alf)) / (2.f * hi32(gaf));
  const float az = fabsf(zf);
  float tf = az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f)));
  if (zf < 0.f) tf = -tf;
  C cs, sn;
  rotcs(tf, cs, sn);
  for (int r = gl; r < m; r += G) {
    const C x = ap[r], y = aq[r];
    ap[r] = fnmac(sn, y, mul(cs, x));
    aq[r] = fmac(sn, x, mul(cs, y));
    const C vx = vp[r], vy = vq[r];
    vp[r] = fnmac(sn, vy, mul(cs, vx));
    vq[r] = fmac(sn, vx, mul(cs, vy));
  }
  return true;
}

template <class C, class RI, int G>
__global__ void __launch_bounds__(1024)
k_jacobi_block(const RI* __restrict__ R, int64_t ldR, const int* __restrict__ m_ptr, int m_max,
               int npl, double* __restrict__ sigma, C* __restrict__ Vout, int ldV, int* status,
               int* sweeps_out, int max_sweeps) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  __shared__ int s_flags[2][16];
  __shared__ float s_red[32];
  __shared__ int s_any;
  __shared__ float s_fro;
  __shared__ int s_cos, s_maxcos[2][16];
  const int m = m_ptr ? *m_ptr : m_max;
  const int NC = (int)cl.num_blocks();
  const int c = (int)cl.block_rank();
  const int MP = 2 * NC * npl;
  if (m < 1 || m > m_max || MP < m || (npl & 1) || npl < 2 || NC < 2 || NC > 16 ||
      (int)blockDim.x < npl * G) {
    if (threadIdx.x == 0 && c == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;  // uniform over the cluster
  }
  const size_t bs = (size_t)npl * m_max;                 // one block: column i at i * m_max
  C* Ab = reinterpret_cast<C*>(smem_raw);                // buffer b at Ab + b * bs
  C* Vb = Ab + 4 * bs;
  int* cid = reinterpret_cast<int*>(Vb + 4 * bs);        // cid[b * npl + i]
  double* allnorm = reinterpret_cast<double*>(cid + ((4 * npl + 1) & ~1));  // [MP]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nt >> 5;

  // power-of-two scaling from max |R| (every CTA reads all of R) and ||R||_F^2 in FP32
  float mx = 0.f, fro = 0.f;
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
  // initial blocks: top = block 2c (buffer 0), bottom = block 2c+1 (buffer 1)
  for (int b = 0; b < 2; ++b) {
    for (int i = 0; i < npl; ++i) {
      const int col = (2 * c + b) * npl + i;
      if (tid == 0) cid[b * npl + i] = col;
      C* a = Ab + b * bs + (size_t)i * m_max;
      C* v = Vb + b * bs + (size_t)i * m_max;
      for (int r = tid; r < m; r += nt) {
        C x = Tr<C>::zero();
        if (col < m && r <= col) {
          x = flush_tiny(pow2s<C>(ld_as<C>(R[r + (int64_t)col * ldR]), -ex));
          const float f = hi32(x);
          fro = fmaf(f, f, fro);
        }
        a[r] = x;
        v[r] = (r == col) ? Tr<C>::one() : Tr<C>::zero();
      }
    }
  }
  // every CTA needs the whole ||A||_F^2: the local parts, read from every CTA after the
  // first cluster barrier (which also makes every CTA's shared memory addressable)
  for (int o = 16; o; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if (lane == 0) s_red[wid] = fro;
  __syncthreads();
  if (tid == 0) {
    float f = 0.f;
    for (int w = 0; w < nwarps; ++w) f += s_red[w];
    s_fro = f;
  }
  cl.sync();
  float frot = 0.f;
  for (int q = 0; q < NC; ++q) frot += *cl.map_shared_rank(&s_fro, q);
  const float tol = ctol<C>(m);
  const float floor_abs = tol * tol * frot;
  const int gid = tid / G, gl = tid % G, ngroups = nt / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  int* flags0 = cl.map_shared_rank(&s_flags[0][0], 0);
  const int half = npl / 2;

  int og = 0;  // outer rounds so far (buffer parity)
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s_rot = 0;
      s_cos = 0;
    }
    __syncthreads();
    int rot = 0;
    float mcos = 0.f;  // largest |cos| of a rotated pair in this sweep (this thread)
    for (int o = 0; o < 2 * NC - 1; ++o, ++og) {
      const int p = og & 1;
      C* TA = Ab + (2 * p) * bs;
      C* TV = Vb + (2 * p) * bs;
      C* BA = Ab + (2 * p + 1) * bs;
      C* BV = Vb + (2 * p + 1) * bs;
      if (o == 0) {
        // pairs inside the top and the bottom block: circle method on npl columns
        for (int k = 0; k < npl - 1; ++k) {
          for (int u = gid; u < npl; u += ngroups) {
            C* XA = u < half ? TA : BA;
            C* XV = u < half ? TV : BV;
            const int i = u < half ? u : u - half;
            int x, y;
            if (i == 0) {
              x = npl - 1;
              y = k;
            } else {
              x = (k + i) % (npl - 1);
              y = (k - i + npl - 1) % (npl - 1);
            }
            rot |= jacobi_pair<C, G>(XA + (size_t)x * m_max, XA + (size_t)y * m_max,
                                     XV + (size_t)x * m_max, XV + (size_t)y * m_max, m, gl, gmask,
                                     tol, floor_abs, mcos);
          }
          __syncthreads();
        }
      }
      // cross pairs (top_u, bottom_{(u+k) mod npl})
      for (int k = 0; k < npl; ++k) {
        for (int u = gid; u < npl; u += ngroups) {
          const int w2 = (u + k) % npl;
          rot |= jacobi_pair<C, G>(TA + (size_t)u * m_max, BA + (size_t)w2 * m_max,
                                   TV + (size_t)u * m_max, BV + (size_t)w2 * m_max, m, gl, gmask,
                                   tol, floor_abs, mcos);
        }
        __syncthreads();
      }
      const bool last = o == 2 * NC - 2;
      if (last) {
        // any rotation in this sweep: one flag per CTA into CTA 0 (read after the barrier)
        if (rot && gl == 0) s_rot = 1;
        if (gl == 0 && mcos > 0.f) atomicMax(&s_cos, __float_as_int(mcos));  // |cos| >= 0
        __syncthreads();
        if (tid == 0) {
          flags0[(sweep & 1) * 16 + c] = s_rot;
          cl.map_shared_rank(&s_maxcos[0][0], 0)[(sweep & 1) * 16 + c] = s_cos;
        }
      }
      // move the blocks (circle method on blocks) into the other parity's buffers
      const int q = 1 - p;
      auto put = [&](int rank, int dst, const C* sA, const C* sV, const int* sc) {
        C* dA = cl.map_shared_rank(Ab, rank) + (size_t)dst * bs;
        C* dV = cl.map_shared_rank(Vb, rank) + (size_t)dst * bs;
        int* dc = cl.map_shared_rank(cid, rank) + dst * npl;
        for (int idx = tid; idx < npl * m; idx += nt) {
          const size_t off = (size_t)(idx / m) * m_max + idx % m;
          dA[off] = sA[off];
          dV[off] = sV[off];
        }
        for (int i = tid; i < npl; i += nt) dc[i] = sc[i];
      };
      const int* Tc = cid + (2 * p) * npl;
      const int* Bc = cid + (2 * p + 1) * npl;
      if (c == 0) {
        put(0, 2 * q, TA, TV, Tc);          // top(0) stays
        put(1, 2 * q, BA, BV, Bc);          // bottom(0) -> top(1)
      } else if (c < NC - 1) {
        put(c + 1, 2 * q, TA, TV, Tc);      // top(c) -> top(c+1)
        put(c - 1, 2 * q + 1, BA, BV, Bc);  // bottom(c) -> bottom(c-1)
      } else {
        put(c - 1, 2 * q + 1, BA, BV, Bc);  // bottom(NC-1) -> bottom(NC-2)
        put(c, 2 * q + 1, TA, TV, Tc);      // top(NC-1) -> bottom(NC-1)
      }
      cl.sync();
    }
    if (tid == 0) {
      int any = 0, mc = 0;
      const int* mc0 = cl.map_shared_rank(&s_maxcos[0][0], 0);
      for (int k = 0; k < NC; ++k) {
        any |= flags0[(sweep & 1) * 16 + k];
        mc = max(mc, mc0[(sweep & 1) * 16 + k]);
      }
      // converged when nothing rotated, or when every rotation of the sweep had
      // |cos| < 1e-7: the coupling left after it is of the order of those squared
      // (quadratic convergence), below the rotation threshold
      s_any = any && __int_as_float(mc) >= kEarlyCos;
    }
    __syncthreads();
    if (s_any == 0) break;
  }
  if (sweep >= max_sweeps && tid == 0 && c == 0 && status) atomicOr(status, DEV_SVD_NOCONV);
  if (tid == 0 && c == 0 && sweeps_out) *sweeps_out = sweep + 1;

  // norms of every column into every CTA, then rank and write the local columns
  const int p = og & 1;
  for (int k = wid; k < 2 * npl; k += nwarps) {
    const C* a = Ab + (2 * p + k / npl) * bs + (size_t)(k % npl) * m_max;
    auto acc = lz(Tr<C>::zero());
    for (int r = lane; r < m; r += 32) acc = lz_fmac(a[r], a[r], acc);
    const C nk = lz_fin(lz_gsum<32>(acc, 0xffffffffu));
    if (lane == 0) {
      const int id = cid[(2 * p + k / npl) * npl + k % npl];
      const double nv = to_f64(nk);
      for (int q = 0; q < NC; ++q) cl.map_shared_rank(allnorm, q)[id] = nv;
    }
  }
  cl.sync();
  for (int k = tid; k < 2 * npl; k += nt) {
    const int b = 2 * p + k / npl, i = k % npl;
    const int id = cid[b * npl + i];
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
    const C* v = Vb + b * bs + (size_t)i * m_max;
    for (int r = 0; r < m; ++r) Vout[r + (size_t)rank * ldV] = v[r];
  }
  cl.sync();  // no CTA leaves while others may still write its shared memory
}

std::mutex g_cl_mu;
int g_cl_ok[2][2][17];  // [type][V in global][NC]: 0 unknown, 1 usable, -1 not usable

}  // namespace

size_t jacobi_cluster_smem(Fmt comp, int m_max, int npl, bool vg) {
  const int nslot = 2 * npl + 4;
  const int P2 = 2 * 16 * npl;  // allnorm holds up to MP doubles
  return (size_t)(vg ? 1 : 2) * nslot * m_max * fmt_bytes(comp) + (size_t)((nslot + 1) & ~1) * 4 +
         (size_t)P2 * sizeof(double) + 16;
}
// V in global memory where A and V together do not fit
bool jacobi_cluster_vg(Fmt comp, int m_max, int npl) {
  return jacobi_cluster_smem(comp, m_max, npl, false) > 200 * 1024;
}

// positions per CTA for a cluster of nc CTAs and this m (0 if it does not fit, even with
// V in global memory)
int jacobi_cluster_npl(Fmt comp, int m_max, int nc) {
  int npl = (m_max + 2 * nc - 1) / (2 * nc);
  if (npl < 2) npl = 2;
  if (npl > 64) return 0;
  return jacobi_cluster_smem(comp, m_max, npl, jacobi_cluster_vg(comp, m_max, npl)) <= 200 * 1024 ? npl : 0;
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

template <class C, class RI, int G, bool VG>
static cudaError_t launch_cl(const void* R, int64_t ldR, const int* m_dev, int m_max, int nc,
                             int npl, double* sigma, void* Vout, int ldV, int* status,
                             int* sweeps_out, void* Vg, int ldVg, cudaStream_t s) {
  auto k = k_jacobi_cluster<C, RI, G, VG>;
  const size_t smem = jacobi_cluster_smem(std::is_same<C, df>::value ? Fmt::DF : Fmt::F64, m_max, npl, VG);
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
    int& ok = g_cl_ok[std::is_same<C, df>::value ? 0 : 1][VG ? 1 : 0][nc];
    if (ok == 0) {
      int nclusters = 0;
      ok = (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0) ? 1 : -1;
      cudaGetLastError();
    }
    if (ok < 0) return cudaErrorNotSupported;
  }
  return cudaLaunchKernelEx(&cfg, k, static_cast<const RI*>(R), ldR, m_dev, m_max, npl, sigma,
                            static_cast<C*>(Vout), ldV, status, sweeps_out, 60, static_cast<C*>(Vg), ldVg);
}

cudaError_t launch_jacobi_cluster(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                                  int m_max, int nc, int npl, double* sigma, void* Vout, int ldV,
                                  int* status, int* sweeps_out, void* Vg, int ldVg, cudaStream_t s) {
  const bool wide = m_max > 128;
  // V in global memory (a scratch of ldVg x m_max) where A and V do not both fit
  const bool vg = jacobi_cluster_vg(comp, m_max, npl);
  if (vg && (!Vg || !wide || ldVg < m_max)) return cudaErrorInvalidValue;
#define TT_CL(C, RI)                                                                               \
  return vg ? launch_cl<C, RI, 32, true>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV, status,  \
                                         sweeps_out, Vg, ldVg, s)                                  \
         : wide ? launch_cl<C, RI, 32, false>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV,      \
                                              status, sweeps_out, nullptr, 0, s)                   \
                : launch_cl<C, RI, 16, false>(R, ldR, m_dev, m_max, nc, npl, sigma, Vout, ldV,      \
                                              status, sweeps_out, nullptr, 0, s)
  if (comp == Fmt::DF && rin == Fmt::DF) TT_CL(df, df);
  if (comp == Fmt::DF && rin == Fmt::F32) TT_CL(df, float);
  if (comp == Fmt::DF && rin == Fmt::F64) TT_CL(df, double);
  if (comp == Fmt::F64 && rin == Fmt::F64) TT_CL(double, double);
#undef TT_CL
  return cudaErrorInvalidValue;
}

}  // namespace tt

namespace tt {

namespace {

std::mutex g_blk_mu;
int g_blk_ok[2][17][8];  // [type][NC][smem bucket of 32 KB]: 0 unknown, 1 usable, -1 not

size_t jacobi_block_smem(Fmt comp, int m_max, int nc, int npl) {
  return (size_t)8 * npl * m_max * fmt_bytes(comp) + (size_t)((4 * npl + 1) & ~1) * 4 +
         (size_t)2 * nc * npl * sizeof(double) + 16;
}

template <class C, class RI, int G>
cudaError_t launch_blk(const void* R, int64_t ldR, const int* m_dev, int m_max, int nc, int npl,
                       size_t smem, double* sigma, void* Vout, int ldV, int* status,
                       int* sweeps_out, cudaStream_t s) {
  auto k = k_jacobi_block<C, RI, G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nc > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  int threads = ((npl * G + 31) / 32) * 32;
  if (threads < 64) threads = 64;
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
  {
    std::lock_guard<std::mutex> lk(g_blk_mu);
    const int bucket = (int)std::min<size_t>(7, smem / (32 * 1024));
    int& ok = g_blk_ok[std::is_same<C, df>::value ? 0 : 1][nc][bucket];
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

}  // namespace

// Cluster size and block width for the block-cyclic kernel: 4 CTAs up to m = 96, else 16
// (measured on GB300 for m = 64, 80, 128, 256 against 2, 4, 8 and 16), falling back to
// the next size whose four block buffers fit in shared memory; 0 if none does.
int jacobi_block_plan(Fmt comp, int m_max, int* npl_out) {
  // "svd.block_nc" forces the cluster size (the block-cyclic order is valid for 2..16 CTAs);
  // other values are ignored
  const int forced_nc = tune_get("svd.block_nc", 0);
  const int forced = forced_nc >= 2 && forced_nc <= 16 ? forced_nc : 0;
  const int pref[4] = {m_max <= 96 ? 4 : 16, m_max <= 96 ? 8 : 8, m_max <= 96 ? 2 : 4, m_max <= 96 ? 16 : 2};
  for (int c = 0; c < 4; ++c) {
    const int nc = forced ? forced : pref[c];
    int npl = (m_max + 2 * nc - 1) / (2 * nc);
    npl += npl & 1;
    if (npl < 2) npl = 2;
    const bool fits = npl * (m_max > 96 ? 32 : 16) <= 1024 &&
                      jacobi_block_smem(comp, m_max, nc, npl) <= 220 * 1024;
    if (fits) {
      *npl_out = npl;
      return nc;
    }
    if (forced) return 0;
  }
  return 0;
}

cudaError_t launch_jacobi_block(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                                int m_max, int nc, int npl, double* sigma, void* Vout, int ldV,
                                int* status, int* sweeps_out, cudaStream_t s) {
  const size_t smem = jacobi_block_smem(comp, m_max, nc, npl);
  // lanes per pair: 16 up to m = 96, else a warp (measured on GB300)
  const bool wide = m_max > 96;
#define TT_BLK(C, RI)                                                                            \
  return wide ? launch_blk<C, RI, 32>(R, ldR, m_dev, m_max, nc, npl, smem, sigma, Vout, ldV,     \
                                      status, sweeps_out, s)                                     \
              : launch_blk<C, RI, 16>(R, ldR, m_dev, m_max, nc, npl, smem, sigma, Vout, ldV,     \
                                      status, sweeps_out, s)
  if (comp == Fmt::DF && rin == Fmt::DF) TT_BLK(df, df);
  if (comp == Fmt::DF && rin == Fmt::F32) TT_BLK(df, float);
  if (comp == Fmt::DF && rin == Fmt::F64) TT_BLK(df, double);
  if (comp == Fmt::F64 && rin == Fmt::F64) TT_BLK(double, double);
#undef TT_BLK
  return cudaErrorInvalidValue;
}

}  // namespace tt
