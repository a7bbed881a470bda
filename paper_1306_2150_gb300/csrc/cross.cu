// Cross approximation of the frequency-space solution (Section 4.2).
//
// Xh[i,j] = (Uh[i,:] . Vh[j,:]) / Lambda[i,j],  Lambda[i,j] = a_i b_j + b_i a_j
// (Eq. flr:div): any entry costs O(r), so a rank-adaptive cross builds
// Xh ~= sum_l d_l C[:,l] R[:,l]^T from one residual row and one residual column
// per step (adaptive cross approximation with partial pivoting):
//   row i*:   rho_j = Xh[i*,j] - sum_l C[i*,l] d_l R[j,l]
//   j* = argmax over unused columns |rho_j| (lowest index on ties), d = rho_j*
//   column:   c_i = (Xh[i,j*] - sum_l C[i,l] d_l R[j*,l]) / d,  R[:,k] = rho / d
//   next row: argmax over unused rows |c_i|
//   ||S_k||^2 += 2 sum_{l<k} d_l d (C_l.c)(R_l.r) + d^2 |c|^2 |r|^2
//   stop after two consecutive steps with |d| |c| |r| <= tol ||S_k||, then a
//   splitmix64-drawn probe of residual entries (restart at a bad probe's row).
// The Gram entries C_l.c and R_l.r are kept for the rounding.
//
// One persistent launch per solve: a thread-block cluster of CS CTAs
// (CS <= 16) splits the index range 0..m-1 into CS contiguous slices of S
// indices.  The CTA keeps its slices of Uh, Vh, of the symbol and of the first
// KS skeleton columns in shared memory (column-major; thread t owns entries
// RPT*t .. RPT*t + RPT - 1, read with one vector load), so a half-step touches
// global memory only for skeleton columns beyond KS.
//
// A half-step: evaluate the owned residual entries; reduce them in the CTA
// (argmax, sum of squares, k dot products with warp shuffles); every CTA then
// pushes its partial -- together with the pivot data its own candidate would
// need next (that index's row of Uh or Vh, of C or R, and its symbol) -- into
// an inbox in the shared memory of every CTA of the cluster with remote
// stores; one cluster barrier; every CTA reduces its inbox in rank order (so
// all take the same decision with the same arithmetic) and reads the winning
// candidate's pivot data from its own shared memory.  Inboxes are
// double-buffered by half-step parity, so one barrier per half-step is enough.
#include <cooperative_groups.h>

#include <climits>
#include <map>
#include <tuple>

#include "lr_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long state, unsigned long long t) {
  unsigned long long z = state + t * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ bool better(T a_abs, int a_idx, T b_abs, int b_idx) {
  return a_abs > b_abs || (a_abs == b_abs && a_idx < b_idx);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T& a, int& i, T& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T oa = __shfl_xor_sync(0xffffffffu, a, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    if (better(oa, oi, a, i)) { a = oa; i = oi; v = ov; }
  }
}

// A CTA's message of one half-step, as 32-bit words (the layout does not
// depend on the field values, so remote copies are plain word copies).
template <typename T>
struct Msg {
  static constexpr int W = (int)sizeof(T) / 4;   // words per value
  static constexpr int ABS = 0, VAL = W, SSQ = 2 * W, CA = 3 * W, CB = 4 * W, IDX = 5 * W;
  static constexpr int HDR = 6 * W;               // header words (IDX padded to a value)
  static constexpr int VEC = HDR;                 // candidate's row of Uh or Vh (r values)
  static constexpr int COEF = VEC + KMAX * W;     // candidate's row of C or R (up to KMAX + 1)
  static constexpr int DOTS = COEF + (KMAX + 1) * W;
  static constexpr int WORDS = DOTS + KMAX * W;
};

template <typename T>
__device__ __forceinline__ T& mval(unsigned* m, int off) { return *reinterpret_cast<T*>(m + off); }
template <typename T>
__device__ __forceinline__ T mval(const unsigned* m, int off) { return *reinterpret_cast<const T*>(m + off); }

template <typename T>
struct Shared {
  T wdots[KMAX][32];       // per-warp dot partials, [l][warp]
  T wsum[32];
  T wabs[32], wval[32];
  int widx[32];
  __align__(16) unsigned out[Msg<T>::WORDS];  // this CTA's message before it is pushed
  T d[KMAX + 1];           // pivot values (identical copy in every CTA)
  T dots[KMAX];            // cluster-reduced dot products of the last half-step
  T gr[KMAX];              // R_l . r of the current step
  T vec[KMAX];             // pivot row of Uh or Vh for the next half-step
  T craw[KMAX + 1];        // pivot row of C or R for the next half-step
  T piv_a, piv_b;          // symbol at the pivot index
  double probe[32];
  int probe_row[32];
  T sumsq, val;
  T norm2;                 // ||S_k||_F^2 of the skeleton
  T rsq;                   // |rho|^2 of the current step
  T delta;                 // pivot value of the current step
  T pfloor;                // pivots at or below are treated as zero (noise floor)
  int idx;
  int flag;
  int win;                 // rank whose candidate won the last reduction
  int small;               // consecutive small terms
};

// Dynamic shared-memory layout (identical in every CTA of the cluster).
// Every cached column has SP = blockDim.x * RPT entries (the CTA's S indices
// plus neutral padding).
template <typename T>
struct Cache {
  unsigned* inbox;  // [2][16][Msg::WORDS]
  T* U;             // SP * r (if cache_uv)
  T* V;
  T* a;             // SP
  T* b;
  T* C;             // SP * KS
  T* R;
  unsigned char* used_r;  // SP
  unsigned char* used_c;
};

template <typename T>
__host__ __device__ constexpr size_t inbox_bytes() {
  return (size_t)2 * 16 * Msg<T>::WORDS * 4;
}

template <typename T>
__device__ __forceinline__ Cache<T> carve(unsigned char* base, int SP, int r, int KS, bool cache_uv) {
  Cache<T> c;
  c.inbox = reinterpret_cast<unsigned*>(base);
  T* p = reinterpret_cast<T*>(base + inbox_bytes<T>());
  c.U = p; p += cache_uv ? (size_t)SP * r : 0;
  c.V = p; p += cache_uv ? (size_t)SP * r : 0;
  c.a = p; p += SP;
  c.b = p; p += SP;
  c.C = p; p += (size_t)SP * KS;
  c.R = p; p += (size_t)SP * KS;
  c.used_r = reinterpret_cast<unsigned char*>(p);
  c.used_c = c.used_r + SP;
  return c;
}

// RPT consecutive entries starting at p (p aligned to RPT * sizeof(T), at
// most 16 bytes per access).
template <typename T, int RPT>
__device__ __forceinline__ void ld_rows(const T* p, T (&x)[RPT]) {
  constexpr int B = RPT * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i) {
      const float4 q = reinterpret_cast<const float4*>(p)[i];
      const T* t = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) x[i * (16 / (int)sizeof(T)) + j] = t[j];
    }
  } else if constexpr (B == 8) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    const T* t = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int j = 0; j < RPT; ++j) x[j] = t[j];
  } else {
    x[0] = p[0];
  }
}

// Own-row entries of column l of a skeleton factor: shared cache for l < KS,
// global memory otherwise.
template <typename T, int RPT>
__device__ __forceinline__ void own_col(const T* Xs, const T* Xg, int SP, int ld, int KS, int l,
                                        const int (&e)[RPT], const bool (&ok)[RPT], T (&x)[RPT]) {
  if (l < KS) {
    ld_rows<T, RPT>(Xs + (size_t)l * SP + RPT * threadIdx.x, x);
  } else {
#pragma unroll
    for (int s = 0; s < RPT; ++s) x[s] = ok[s] ? __ldcg(&Xg[e[s] + (size_t)l * ld]) : T(0);
  }
}

template <typename T> __device__ __forceinline__ T ratio(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float ratio<float>(float a, float b) { return __fdividef(a, b); }

// Sum over the warp of a[i], i < W, for every i at once (recursive halving:
// at each stage a lane keeps one half of its vector and receives the
// partner's copy of that half).  Afterwards every lane L holds the sum for
// index L mod W.  W - 1 + log2(32/W) shuffles instead of 5 W; the addition
// pattern is fixed, so every CTA gets the same bits.
template <typename T, int W>
__device__ __forceinline__ T warp_transpose_sum(T (&a)[W], int lane) {
#pragma unroll
  for (int h = W / 2; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? a[i] : a[i + h];
      const T keep = up ? a[i + h] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  T x = a[0];
#pragma unroll
  for (int o = W; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Warp partials of dots[l] = sum over own rows of X[row, l] v[row] for
// l in [l0, l0 + W) with l < k.
template <typename T, int RPT, int W>
__device__ __forceinline__ void warp_dots(const T (&v)[RPT], const bool (&ok)[RPT], const int (&e)[RPT],
                                          const T* Xs, const T* Xg, int SP, int ld, int KS, int l0, int k,
                                          Shared<T>& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T a[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    a[i] = T(0);
    const int l = l0 + i;
    if (l < k) {
      T x[RPT];
      own_col<T, RPT>(Xs, Xg, SP, ld, KS, l, e, ok, x);
#pragma unroll
      for (int s = 0; s < RPT; ++s) a[i] += x[s] * v[s];
    }
  }
  const T x = warp_transpose_sum<T, W>(a, lane);
  if (lane < W && l0 + lane < k) sh.wdots[l0 + lane][warp] = x;
}

// Where the pivot data for the next half-step comes from: the factor F (Uh
// or Vh, r columns) and the skeleton factor X (C or R, kn columns).
template <typename T>
struct NextSide {
  const T* Fs;   // shared cache of F (if cached)
  const T* Fg;   // F in global memory
  const T* Xs;   // shared cache of X (columns < KS)
  const T* Xg;   // X in global memory
  int kn;
};

// Reduce over the CTA and the cluster (see the file comment): argmax |v|
// among candidates (lowest index on ties), sum of v^2 and, for l < k,
// dots[l] = sum v * Xd[own row, l].  Results: sh.idx (-1 if no candidate),
// sh.val, sh.sumsq, sh.dots, and the winner's pivot data sh.vec, sh.craw,
// sh.piv_a, sh.piv_b from nx.  v must be 0 for rows that are not owned.
template <typename T, int RPT>
__device__ __forceinline__ void cluster_reduce(cg::cluster_group& cl, int CS, int SP, int row0, int r,
                                               int KS, bool cache_uv, int ld, const Cache<T>& cc,
                                               const T (&v)[RPT], const bool (&ok)[RPT],
                                               const bool (&cand)[RPT], const int (&e)[RPT], const T* Xds,
                                               const T* Xdg, int k, const NextSide<T>& nx, int& par,
                                               Shared<T>& sh) {
  using M = Msg<T>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
  const int q = (int)cl.block_rank();
  T babs = T(-1), bval = T(0), ssq = T(0);
  int bidx = INT_MAX;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    ssq += v[s] * v[s];
    if (cand[s]) {
      const T av = fabs(v[s]);
      if (better(av, e[s], babs, bidx)) { babs = av; bidx = e[s]; bval = v[s]; }
    }
  }
  warp_argmax(babs, bidx, bval);
  ssq = warp_sum(ssq);
  // 16-wide chunks: 16 shuffles per chunk, and a 16-entry register buffer
  // keeps the register pressure low when a thread owns several rows.
  if (k > 0 && k <= 8) warp_dots<T, RPT, 8>(v, ok, e, Xds, Xdg, SP, ld, KS, 0, k, sh);
  else
    for (int l0 = 0; l0 < k; l0 += 16) warp_dots<T, RPT, 16>(v, ok, e, Xds, Xdg, SP, ld, KS, l0, k, sh);
  if (lane == 0) { sh.wabs[warp] = babs; sh.widx[warp] = bidx; sh.wval[warp] = bval; sh.wsum[warp] = ssq; }
  __syncthreads();
  // CTA reduction into this CTA's message.
  if (warp == 0) {
    T a = lane < NW ? sh.wabs[lane] : T(-1);
    int i = lane < NW ? sh.widx[lane] : INT_MAX;
    T vv = lane < NW ? sh.wval[lane] : T(0);
    T ss = lane < NW ? sh.wsum[lane] : T(0);
    warp_argmax(a, i, vv);
    ss = warp_sum(ss);
    if (lane == 0) {
      mval<T>(sh.out, M::ABS) = a;
      mval<T>(sh.out, M::VAL) = vv;
      mval<T>(sh.out, M::SSQ) = ss;
      sh.out[M::IDX] = (unsigned)i;
    }
  }
  // dots: one l per half-warp of 16 lanes, lane w reads warp w (NW <= 16)
  for (int base = warp * 32; base < k * 16; base += (int)blockDim.x) {
    const int t = base + lane, l = t >> 4, w = t & 15;
    T x = (t < k * 16 && w < NW) ? sh.wdots[l][w] : T(0);
    x += __shfl_xor_sync(0xffffffffu, x, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    if (w == 0 && t < k * 16) mval<T>(sh.out, M::DOTS + l * M::W) = x;
  }
  __syncthreads();
  // The pivot data the CTA's own candidate would need next.
  {
    const int ci = (int)sh.out[M::IDX];
    if (ci != INT_MAX) {
      const int loc = ci - row0;
      if (tid < r) {
        mval<T>(sh.out, M::VEC + tid * M::W) =
            cache_uv ? nx.Fs[(size_t)tid * SP + loc] : nx.Fg[ci + (size_t)tid * ld];
      } else if (tid >= KMAX && tid < KMAX + nx.kn) {
        const int l = tid - KMAX;
        mval<T>(sh.out, M::COEF + l * M::W) =
            l < KS ? nx.Xs[(size_t)l * SP + loc] : __ldcg(&nx.Xg[ci + (size_t)l * ld]);
      } else if (tid == 2 * KMAX + 1) {
        mval<T>(sh.out, M::CA) = cc.a[loc];
        mval<T>(sh.out, M::CB) = cc.b[loc];
      }
    }
  }
  __syncthreads();
  // Push the live words of the message into slot q of every CTA's inbox.
  {
    const int nv = r * M::W, nc = nx.kn * M::W, nd = k * M::W;
    const int live = M::HDR + nv + nc + nd;
    unsigned* slot = cc.inbox + ((size_t)par * 16 + q) * M::WORDS;
    for (int i = tid; i < CS * live; i += (int)blockDim.x) {
      const int dst = i / live;
      int w = i - dst * live;
      int off;
      if (w < M::HDR) off = w;
      else if ((w -= M::HDR) < nv) off = M::VEC + w;
      else if ((w -= nv) < nc) off = M::COEF + w;
      else off = M::DOTS + (w - nc);
      *cl.map_shared_rank(slot + off, dst) = sh.out[off];
    }
  }
  cl.sync();
  // Reduce the inbox (local shared memory) in rank order.
  const unsigned* box = cc.inbox + (size_t)par * 16 * M::WORDS;
  if (warp == 0) {
    T a = T(-1), vv = T(0), ss = T(0);
    int i = INT_MAX, src = lane;
    if (lane < CS) {
      const unsigned* m = box + (size_t)lane * M::WORDS;
      a = mval<T>(m, M::ABS); vv = mval<T>(m, M::VAL); ss = mval<T>(m, M::SSQ); i = (int)m[M::IDX];
    }
    // argmax carrying the source rank along with the value
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T oa = __shfl_xor_sync(0xffffffffu, a, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      const T ov = __shfl_xor_sync(0xffffffffu, vv, o);
      const int os = __shfl_xor_sync(0xffffffffu, src, o);
      if (better(oa, oi, a, i)) { a = oa; i = oi; vv = ov; src = os; }
    }
    ss = warp_sum(ss);
    if (lane == 0) {
      const bool none = i == INT_MAX || a < T(0);
      sh.idx = none ? -1 : i;
      sh.val = vv;
      sh.sumsq = ss;
      sh.win = none ? -1 : src;
    }
  }
  for (int base = warp * 32; base < k * 16; base += (int)blockDim.x) {
    const int t = base + lane, l = t >> 4, qq = t & 15;
    T x = (t < k * 16 && qq < CS) ? mval<T>(box + (size_t)qq * M::WORDS, M::DOTS + l * M::W) : T(0);
    x += __shfl_xor_sync(0xffffffffu, x, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    if (qq == 0 && t < k * 16) sh.dots[l] = x;
  }
  __syncthreads();
  // The winner's pivot data for the next half-step.
  const int win = sh.win;
  if (win >= 0) {
    const unsigned* m = box + (size_t)win * M::WORDS;
    if (tid < r) sh.vec[tid] = mval<T>(m, M::VEC + tid * M::W);
    else if (tid >= KMAX && tid < KMAX + nx.kn) sh.craw[tid - KMAX] = mval<T>(m, M::COEF + (tid - KMAX) * M::W);
    else if (tid == 2 * KMAX + 1) { sh.piv_a = mval<T>(m, M::CA); sh.piv_b = mval<T>(m, M::CB); }
  }
  __syncthreads();
  par ^= 1;
}

// Residual entries of the owned indices for a half-step at the pivot whose
// data is in sh: out[s] = (sum_al vec[al] F[own, al]) / (pa * b_own + pb * a_own)
//                         - sum_l craw[l] d[l] X[own, l].
template <typename T, int RPT>
__device__ __forceinline__ void eval_entries(const Shared<T>& sh, const Cache<T>& cc, const T* Fs,
                                             const T* __restrict__ Fg, const T* Xs, const T* Xg, int SP,
                                             int ld, int r, int k, int KS, bool cache_uv, const int (&e)[RPT],
                                             const bool (&ok)[RPT], T (&out)[RPT]) {
  const int base = RPT * threadIdx.x;
  T num[RPT];
#pragma unroll
  for (int s = 0; s < RPT; ++s) num[s] = T(0);
  for (int al = 0; al < r; ++al) {
    T f[RPT];
    if (cache_uv) {
      ld_rows<T, RPT>(Fs + (size_t)al * SP + base, f);
    } else {
#pragma unroll
      for (int s = 0; s < RPT; ++s) f[s] = ok[s] ? Fg[e[s] + (size_t)al * ld] : T(0);
    }
    const T w = sh.vec[al];
#pragma unroll
    for (int s = 0; s < RPT; ++s) num[s] += w * f[s];
  }
  T av[RPT], bv[RPT];
  ld_rows<T, RPT>(cc.a + base, av);
  ld_rows<T, RPT>(cc.b + base, bv);
  const T pa = sh.piv_a, pb = sh.piv_b;
#pragma unroll
  for (int s = 0; s < RPT; ++s) out[s] = ratio<T>(num[s], pa * bv[s] + pb * av[s]);
  for (int l = 0; l < k; ++l) {
    T x[RPT];
    own_col<T, RPT>(Xs, Xg, SP, ld, KS, l, e, ok, x);
    const T c = sh.craw[l] * sh.d[l];
#pragma unroll
    for (int s = 0; s < RPT; ++s) out[s] -= c * x[s];
  }
#pragma unroll
  for (int s = 0; s < RPT; ++s)
    if (!ok[s]) out[s] = T(0);
}

template <typename T, int RPT>
__global__ void __launch_bounds__(512, 1) cross_kernel(CrossArgs<T> A, int KS, int cache_uv_i) {
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int CS = (int)cl.num_blocks();
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int m = A.m, r = A.r, ld = A.ld;
  const int S = (m + CS - 1) / CS;
  const int SP = NT * RPT;  // >= S
  const int row0 = min(m, q * S), row1 = min(m, row0 + S);
  const bool cache_uv = cache_uv_i != 0;
  const T tol2 = (T)(A.tol * A.tol);

  __shared__ Shared<T> sh;
  extern __shared__ __align__(16) unsigned char dyn[];
  const Cache<T> cc = carve<T>(dyn, SP, r, KS, cache_uv);

  // Fill the caches (neutral values past the end of the index range).
  for (int i = tid; i < SP; i += NT) {
    const int e = row0 + i;
    const bool in = e < row1;
    cc.a[i] = in ? A.a[e] : T(1);
    cc.b[i] = in ? A.b[e] : T(1);
    cc.used_r[i] = 0;
    cc.used_c[i] = 0;
    if (cache_uv)
      for (int al = 0; al < r; ++al) {
        cc.U[(size_t)al * SP + i] = in ? A.Uh[e + (size_t)al * ld] : T(0);
        cc.V[(size_t)al * SP + i] = in ? A.Vh[e + (size_t)al * ld] : T(0);
      }
  }
  for (int i = tid; i < SP * KS; i += NT) { cc.C[i] = T(0); cc.R[i] = T(0); }
  if (tid == 0) { sh.norm2 = T(0); sh.small = 0; sh.pfloor = T(0); }
  __syncthreads();
  // Every CTA must be running before anyone pushes into its inbox.
  cl.sync();

  int e[RPT];
  bool ok[RPT], cand[RPT];
  T v[RPT], score[RPT];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    e[s] = row0 + RPT * tid + s;
    ok[s] = e[s] < row1;
  }
  const NextSide<T> to_row{cc.U, A.Uh, cc.C, A.C, 0};   // kn is set per use
  const NextSide<T> to_col{cc.V, A.Vh, cc.R, A.R, 0};
  const T a0 = A.a[0], b0 = A.b[0];
  // Start score ||Uh[i]||^2 / Lambda[i,0]^2 (an upper-bound proxy of row size).
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    score[s] = T(0);
    if (ok[s]) {
      const int loc = RPT * tid + s;
      T acc = T(0);
      for (int al = 0; al < r; ++al) {
        const T u = cache_uv ? cc.U[(size_t)al * SP + loc] : A.Uh[e[s] + (size_t)al * ld];
        acc += u * u;
      }
      const T lam0 = cc.a[loc] * b0 + cc.b[loc] * a0;
      score[s] = acc / (lam0 * lam0);
    }
    cand[s] = ok[s];
  }
  int par = 0;
  NextSide<T> nx = to_row;
  cluster_reduce<T, RPT>(cl, CS, SP, row0, r, KS, cache_uv, ld, cc, score, ok, cand, e, cc.C, A.C, 0, nx, par, sh);
  int istar = sh.idx;

  int k = 0, probe_rounds = 0, zero_rows = 0;
  int converged = 0;
  while (k < A.kcap && istar >= 0) {
    // ---------------- row half-step at istar (pivot data already in sh)
    eval_entries<T, RPT>(sh, cc, cc.V, A.Vh, cc.R, A.R, SP, ld, r, k, KS, cache_uv, e, ok, v);
#pragma unroll
    for (int s = 0; s < RPT; ++s) cand[s] = ok[s] && cc.used_c[RPT * tid + s] == 0;
    if (istar >= row0 && istar < row1 && tid == 0) cc.used_r[istar - row0] = 1;
    nx = to_col;
    nx.kn = k;
    cluster_reduce<T, RPT>(cl, CS, SP, row0, r, KS, cache_uv, ld, cc, v, ok, cand, e, cc.R, A.R, k, nx, par, sh);
    const int jstar = sh.idx;
    if (tid == 0) {
      const T dv = jstar >= 0 ? sh.val : T(0);
      // A pivot far below the working precision's rounding noise (relative to
      // the first pivot) is a zero row: dividing by it would only overflow.
      sh.flag = !(fabs(dv) > sh.pfloor);
      sh.delta = dv;
      sh.rsq = sh.sumsq;
      if (jstar >= row0 && jstar < row1) cc.used_c[jstar - row0] = 1;
    }
    __syncthreads();
    if (sh.flag) {
      // The row is already represented exactly: move to the best-scored
      // unused row (rows are marked used above).
      ++zero_rows;
#pragma unroll
      for (int s = 0; s < RPT; ++s) cand[s] = ok[s] && cc.used_r[RPT * tid + s] == 0;
      nx = to_row;
      nx.kn = k;
      cluster_reduce<T, RPT>(cl, CS, SP, row0, r, KS, cache_uv, ld, cc, score, ok, cand, e, cc.C, A.C, 0, nx, par,
                             sh);
      if (zero_rows > A.max_zero_rows || sh.idx < 0) { converged = 1; break; }
      istar = sh.idx;
      continue;
    }
    // ---------------- column half-step at jstar
    const T tdelta = sh.delta;
    for (int l = tid; l < k; l += NT) sh.gr[l] = sh.dots[l] / tdelta;
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      if (!ok[s]) continue;
      const T rv = v[s] / tdelta;
      if (k < KS) cc.R[(size_t)k * SP + RPT * tid + s] = rv;
      A.R[e[s] + (size_t)k * ld] = rv;
    }
    eval_entries<T, RPT>(sh, cc, cc.U, A.Uh, cc.C, A.C, SP, ld, r, k, KS, cache_uv, e, ok, v);
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      v[s] = v[s] / tdelta;
      cand[s] = ok[s] && cc.used_r[RPT * tid + s] == 0;
      if (!ok[s]) continue;
      if (k < KS) cc.C[(size_t)k * SP + RPT * tid + s] = v[s];
      A.C[e[s] + (size_t)k * ld] = v[s];
    }
    // The pivot value is appended only now: the column evaluation above
    // used d[0..k) and the next row step needs d[0..k].
    __syncthreads();
    if (tid == 0) sh.d[k] = tdelta;
    nx = to_row;
    nx.kn = k + 1;   // the next row step needs the new column k of C
    cluster_reduce<T, RPT>(cl, CS, SP, row0, r, KS, cache_uv, ld, cc, v, ok, cand, e, cc.C, A.C, k, nx, par, sh);
    const int inext = sh.idx;
    // ---------------- bookkeeping (thread 0 of every CTA, same arithmetic)
    if (tid == 0) {
      const T delta = sh.delta;
      const T csq = sh.sumsq;
      // |r|^2 = |row|^2 / delta^2 <= m (delta is the row's largest entry);
      // divided twice so that delta^2 never underflows.
      const T rr = (sh.rsq / delta) / delta;
      T cs = T(0);
      for (int l = 0; l < k; ++l) cs += sh.d[l] * sh.dots[l] * sh.gr[l];
      const T term2 = csq * sh.rsq;                   // |d|^2 |c|^2 |r|^2
      sh.norm2 += T(2) * delta * cs + term2;
      sh.small = (term2 <= tol2 * sh.norm2) ? sh.small + 1 : 0;
      if (k == 0) sh.pfloor = fabs(delta) * (T)(sizeof(T) == 4 ? 1e-9 : 1e-20);
      if (q == 0) {
        A.GC[k + (size_t)k * A.kcap] = (double)csq;
        A.GR[k + (size_t)k * A.kcap] = (double)rr;
        A.d[k] = (double)delta;
        A.I[k] = istar;
        A.J[k] = jstar;
      }
    }
    if (q == 0)
      for (int l = tid; l < k; l += NT) {
        const double gc = (double)sh.dots[l], gr = (double)sh.gr[l];
        A.GC[l + (size_t)k * A.kcap] = gc;
        A.GC[k + (size_t)l * A.kcap] = gc;
        A.GR[l + (size_t)k * A.kcap] = gr;
        A.GR[k + (size_t)l * A.kcap] = gr;
      }
    __syncthreads();
    ++k;
    if (sh.small >= 2) {
      if (probe_rounds >= A.max_probe_rounds || A.probes <= 0) { converged = 1; break; }
      // Residual probes at splitmix64-drawn entries; probe p on warp p mod
      // (warps per CTA), the same arithmetic in every CTA.
      const int P = A.probes < 32 ? A.probes : 32;
      for (int p = warp; p < P; p += NT >> 5) {
        const unsigned long long z = splitmix64_at(A.seed + (unsigned long long)probe_rounds,
                                                   (unsigned long long)(p + 1));
        const int pi = (int)((z >> 32) % (unsigned long long)m);
        const int pj = (int)((z & 0xFFFFFFFFULL) % (unsigned long long)m);
        double num = 0.0, sk = 0.0;
        for (int al = lane; al < r; al += 32)
          num += (double)A.Uh[pi + (size_t)al * ld] * (double)A.Vh[pj + (size_t)al * ld];
        for (int l = lane; l < k; l += 32)
          sk += (double)__ldcg(&A.C[pi + (size_t)l * ld]) * (double)sh.d[l] *
                (double)__ldcg(&A.R[pj + (size_t)l * ld]);
        num = warp_sum(num);
        sk = warp_sum(sk);
        const double den = (double)A.a[pi] * (double)A.b[pj] + (double)A.b[pi] * (double)A.a[pj];
        if (lane == 0) { sh.probe[p] = fabs(num / den - sk); sh.probe_row[p] = pi; }
      }
      __syncthreads();
      if (tid == 0) {
        double worst = -1.0;
        int wrow = -1;
        for (int p = 0; p < P; ++p)
          if (sh.probe[p] > worst) { worst = sh.probe[p]; wrow = sh.probe_row[p]; }
        const double n2 = (double)sh.norm2;
        sh.flag = worst <= A.tol * sqrt(n2 > 0.0 ? n2 : 0.0) ? -1 : wrow;
        if (sh.flag >= 0) sh.small = 0;
      }
      __syncthreads();
      ++probe_rounds;
      const int bad_row = sh.flag;
      if (bad_row < 0) { converged = 1; break; }
      // Restart at the bad probe's row if unused, else at the best unused
      // score; the owner's answer reaches every CTA through the reduction.
      T bump[RPT];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const bool unused = ok[s] && cc.used_r[RPT * tid + s] == 0;
        cand[s] = unused;
        bump[s] = (unused && e[s] == bad_row) ? T(INFINITY) : score[s];
      }
      nx = to_row;
      nx.kn = k;
      cluster_reduce<T, RPT>(cl, CS, SP, row0, r, KS, cache_uv, ld, cc, bump, ok, cand, e, cc.C, A.C, 0, nx, par,
                             sh);
      istar = sh.idx;
      if (istar < 0) { converged = 1; break; }
      continue;
    }
    istar = inext;
    if (istar < 0) { converged = 1; break; }
  }
  // No CTA may exit while another can still write into its shared memory.
  cl.sync();
  if (q == 0 && tid == 0) {
    A.st->k = k;
    A.st->converged = converged;
    A.st->probe_rounds = probe_rounds;
    A.st->zero_rows = zero_rows;
    A.st->norm2 = (double)sh.norm2;
  }
}

// Per-kernel launch facts that do not change during a process: set the
// attributes and query the static shared memory once, not before every launch.
struct KernelFacts {
  bool ready = false;
  cudaError_t err = cudaSuccess;
  int optin = 0;
  size_t static_smem = 0;
};

template <typename T, int RPT>
static KernelFacts& cross_facts() {
  static KernelFacts f;
  if (!f.ready) {
    auto kern = cross_kernel<T, RPT>;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&f.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    f.err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (f.err == cudaSuccess) f.err = cudaFuncGetAttributes(&fa, kern);
    if (f.err == cudaSuccess) {
      f.static_smem = fa.sharedSizeBytes;
      f.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   f.optin - (int)fa.sharedSizeBytes);
    }
    f.ready = true;
  }
  return f;
}

// Clusters of a configuration that fit on the device (memoised).
static std::map<std::tuple<const void*, int, int, size_t>, int>& cluster_fit_cache() {
  static std::map<std::tuple<const void*, int, int, size_t>, int> c;
  return c;
}

template <typename T, int RPT>
static cudaError_t launch_cross_rpt(const CrossArgs<T>& a, int cs, int nt, cudaStream_t st) {
  auto kern = cross_kernel<T, RPT>;
  const KernelFacts& f = cross_facts<T, RPT>();
  if (f.err != cudaSuccess) return f.err;
  cudaError_t e;
  // Shared-memory budget: inboxes, symbol slices and flags always, Uh/Vh
  // slices if they fit in half of what is left, then as many skeleton
  // columns as fit.
  const long long SP = (long long)nt * RPT;
  const long long w = (long long)sizeof(T);
  const long long budget = (long long)f.optin - (long long)f.static_smem - 1024;
  const long long fixed = (long long)inbox_bytes<T>() + 2LL * SP * w + 2LL * SP + 64;
  if (fixed > budget) return cudaErrorInvalidConfiguration;
  const long long uv = 2LL * SP * a.r * w;
  const bool cache_uv = uv <= (budget - fixed) / 2;
  const long long left = budget - fixed - (cache_uv ? uv : 0);
  long long KS = left / (2LL * SP * w);
  if (KS > a.kcap) KS = a.kcap;
  if (KS < 0) KS = 0;
  const size_t dsmem = (size_t)(fixed + (cache_uv ? uv : 0) + 2LL * SP * KS * w);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(nt, 1, 1);
  cfg.dynamicSmemBytes = dsmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const auto key = std::make_tuple((const void*)kern, cs, nt, dsmem);
  auto it = cluster_fit_cache().find(key);
  int nclusters = 0;
  if (it == cluster_fit_cache().end()) {
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    cluster_fit_cache()[key] = nclusters;
  } else {
    nclusters = it->second;
  }
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  return cudaLaunchKernelEx(&cfg, kern, a, (int)KS, cache_uv ? 1 : 0);
}

// Rows per thread RPT (a power of two) and threads per CTA for S indices:
// about four rows per thread, 160 to 512 threads (threads up to 2*KMAX + 1
// carry pivot data); more rows per thread only when S exceeds 512 * 4.
static void cross_shape(int S, int* nt, int* rpt) {
  int r = 1;
  while (r < 4 && r * 160 < S) r *= 2;
  while (r < 16 && r * 512 < S) r *= 2;
  int t = (S + r - 1) / r;
  t = (t + 31) / 32 * 32;
  if (t < 160) t = 160;
  *nt = t;
  *rpt = r;
}

template <typename T>
cudaError_t launch_cross(const CrossArgs<T>& a, int cluster_size, cudaStream_t st, int* used_cluster) {
  // Largest index range a CTA may own: 512 threads x 16 rows.
  const int cs_min = (a.m + 512 * 16 - 1) / (512 * 16);
  int cs = cluster_size;
  if (cs <= 0) {
    cs = (a.m + 1023) / 1024;
    if (cs > 16) cs = 16;
  }
  if (cs < cs_min) cs = cs_min;
  if (cs < 1) cs = 1;
  if (cs > 16) return cudaErrorInvalidValue;
  cudaError_t e = cudaErrorInvalidConfiguration;
  for (; cs >= cs_min && cs >= 1; cs = (cs > 8 ? 8 : cs - 1)) {
    const int S = (a.m + cs - 1) / cs;
    int nt, rpt;
    cross_shape(S, &nt, &rpt);
    if (rpt == 1) e = launch_cross_rpt<T, 1>(a, cs, nt, st);
    else if (rpt == 2) e = launch_cross_rpt<T, 2>(a, cs, nt, st);
    else if (rpt == 4) e = launch_cross_rpt<T, 4>(a, cs, nt, st);
    else if (rpt == 8) e = launch_cross_rpt<T, 8>(a, cs, nt, st);
    else e = launch_cross_rpt<T, 16>(a, cs, nt, st);
    if (e == cudaSuccess) { if (used_cluster) *used_cluster = cs; return e; }
    if (e != cudaErrorInvalidConfiguration && e != cudaErrorInvalidClusterSize &&
        e != cudaErrorLaunchOutOfResources)
      return e;
    cudaGetLastError();  // clear the launch-configuration error and retry smaller
  }
  return e;
}

template cudaError_t launch_cross<double>(const CrossArgs<double>&, int, cudaStream_t, int*);
template cudaError_t launch_cross<float>(const CrossArgs<float>&, int, cudaStream_t, int*);

}  // namespace lrp
