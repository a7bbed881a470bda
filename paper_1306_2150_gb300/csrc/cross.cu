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
// The Gram entries C_l.c and R_l.r are kept (FP64) for the rounding.
//
// One persistent launch per solve: a thread-block cluster of CS CTAs
// (CS <= 16) splits the index range 0..m-1 into CS contiguous slices; each
// thread owns up to RPT indices of its CTA's slice for both the row and the
// column side.  A half-step is: broadcast row/coefficient vectors, evaluate the
// owned residual entries, reduce (argmax, sum of squares, k dot products) with
// warp shuffles and shared memory, publish the CTA partial in shared memory,
// one cluster barrier, then every CTA reads all partials through distributed
// shared memory in rank order, so every CTA takes the same decision with the
// same arithmetic.  Partials are double-buffered by half-step parity, which
// makes one barrier per half-step enough.
#include <cooperative_groups.h>

#include <climits>

#include "lr_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

template <typename T>
struct Partial {
  double sumsq;
  double dots[KMAX];
  T absmax;
  T val;
  int idx;
  int pad;
};

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

struct Shared {
  double wdots[32][KMAX];
  double wsum[32];
  double d[KMAX];        // pivot values (identical copy in every CTA)
  double dots[KMAX];     // cluster-reduced dot products of the last half-step
  double gc[KMAX];       // C_l . c of the current step
  double gr[KMAX];       // R_l . r of the current step
  double sumsq, val;
  int idx;
  int flag;
};

// Reduce over the CTA and then the cluster: argmax |v| among candidates
// (lowest index on ties), sum of v^2 and dots[l] = sum v * X[:, l], l < k.
// Results land in sh.idx (-1 if no candidate), sh.val, sh.sumsq, sh.dots.
template <typename T, int RPT>
__device__ __forceinline__ void cluster_reduce(cg::cluster_group& cl, int CS, const T (&v)[RPT],
                                               const bool (&ok)[RPT], const bool (&cand)[RPT],
                                               const int (&e)[RPT], const T* __restrict__ X, int ld,
                                               int k, Partial<T>* xb, int& par, Shared& sh,
                                               T* wabs, T* wval, int* widx) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
  T babs = T(-1), bval = T(0), ssq = T(0);
  int bidx = INT_MAX;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    if (!ok[s]) continue;
    ssq += v[s] * v[s];
    if (cand[s]) {
      const T av = fabs(v[s]);
      if (better(av, e[s], babs, bidx)) { babs = av; bidx = e[s]; bval = v[s]; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T oa = __shfl_xor_sync(0xffffffffu, babs, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    const T ov = __shfl_xor_sync(0xffffffffu, bval, o);
    if (better(oa, oi, babs, bidx)) { babs = oa; bidx = oi; bval = ov; }
  }
  ssq = warp_sum(ssq);
  for (int l = 0; l < k; ++l) {
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (ok[s]) acc += X[e[s] + (size_t)l * ld] * v[s];
    acc = warp_sum(acc);
    if (lane == 0) sh.wdots[warp][l] = (double)acc;
  }
  if (lane == 0) { wabs[warp] = babs; widx[warp] = bidx; wval[warp] = bval; sh.wsum[warp] = (double)ssq; }
  __syncthreads();
  Partial<T>& P = xb[par];
  if (tid == 0) {
    T ba = T(-1), bv = T(0);
    int bi = INT_MAX;
    double ss = 0.0;
    for (int w = 0; w < NW; ++w) {
      if (better(wabs[w], widx[w], ba, bi)) { ba = wabs[w]; bi = widx[w]; bv = wval[w]; }
      ss += sh.wsum[w];
    }
    P.absmax = ba; P.idx = bi; P.val = bv; P.sumsq = ss;
  }
  for (int l = tid; l < k; l += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < NW; ++w) acc += sh.wdots[w][l];
    P.dots[l] = acc;
  }
  cl.sync();
  if (tid == 0) {
    T ba = T(-1), bv = T(0);
    int bi = INT_MAX;
    double ss = 0.0;
    for (int rk = 0; rk < CS; ++rk) {
      const Partial<T>* Q = cl.map_shared_rank(&xb[par], rk);
      const T qa = Q->absmax;
      const int qi = Q->idx;
      if (better(qa, qi, ba, bi)) { ba = qa; bi = qi; bv = Q->val; }
      ss += Q->sumsq;
    }
    sh.idx = (bi == INT_MAX || ba < T(0)) ? -1 : bi;
    sh.val = (double)bv;
    sh.sumsq = ss;
  }
  for (int l = tid; l < k; l += blockDim.x) {
    double acc = 0.0;
    for (int rk = 0; rk < CS; ++rk) acc += cl.map_shared_rank(&xb[par], rk)->dots[l];
    sh.dots[l] = acc;
  }
  __syncthreads();
  par ^= 1;
}

template <typename T, int RPT>
__global__ void __launch_bounds__(1024, 1) cross_kernel(CrossArgs<T> A) {
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int CS = (int)cl.num_blocks();
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int m = A.m, r = A.r, ld = A.ld;
  const int S = (m + CS - 1) / CS;
  const int row0 = min(m, q * S), row1 = min(m, row0 + S);

  __shared__ Partial<T> xb[2];
  __shared__ Shared sh;
  __shared__ T wabs[32], wval[32];
  __shared__ int widx[32];
  __shared__ T s_vec[KMAX];
  __shared__ T s_coef[KMAX];
  __shared__ double s_probe[32];
  __shared__ int s_probe_row[32];
  extern __shared__ unsigned char used[];  // [0, S): rows, [S, 2S): columns
  unsigned char* used_r = used;
  unsigned char* used_c = used + S;

  for (int i = tid; i < 2 * S; i += NT) used[i] = 0;

  int e[RPT];
  bool ok[RPT], cand[RPT];
  T v[RPT], score[RPT];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    e[s] = row0 + tid + s * NT;
    ok[s] = e[s] < row1;
  }
  const T a0 = A.a[0], b0 = A.b[0];
  // Start score ||Uh[i]||^2 / Lambda[i,0]^2 (an upper-bound proxy of row size).
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    score[s] = T(0);
    if (ok[s]) {
      T acc = T(0);
      for (int al = 0; al < r; ++al) {
        const T u = A.Uh[e[s] + (size_t)al * ld];
        acc += u * u;
      }
      const T lam0 = A.a[e[s]] * b0 + A.b[e[s]] * a0;
      score[s] = acc / (lam0 * lam0);
    }
    cand[s] = ok[s];
  }
  __syncthreads();
  int par = 0;
  cluster_reduce<T, RPT>(cl, CS, score, ok, cand, e, A.C, ld, 0, xb, par, sh, wabs, wval, widx);
  int istar = sh.idx;

  double norm2 = 0.0;
  int k = 0, small = 0, probe_rounds = 0, zero_rows = 0;
  int converged = 0;
  while (k < A.kcap && istar >= 0) {
    // ---------------- row half-step at istar
    for (int al = tid; al < r; al += NT) s_vec[al] = A.Uh[istar + (size_t)al * ld];
    for (int l = tid; l < k; l += NT) s_coef[l] = (T)((double)__ldcg(&A.C[istar + (size_t)l * ld]) * sh.d[l]);
    __syncthreads();
    {
      const T ai = A.a[istar], bi = A.b[istar];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        v[s] = T(0);
        if (!ok[s]) continue;
        const int j = e[s];
        T num = T(0);
        for (int al = 0; al < r; ++al) num += s_vec[al] * A.Vh[j + (size_t)al * ld];
        T x = num / (ai * A.b[j] + bi * A.a[j]);
        for (int l = 0; l < k; ++l) x -= s_coef[l] * A.R[j + (size_t)l * ld];
        v[s] = x;
        cand[s] = used_c[j - row0] == 0;
      }
    }
    if (istar >= row0 && istar < row1 && tid == 0) used_r[istar - row0] = 1;
    cluster_reduce<T, RPT>(cl, CS, v, ok, cand, e, A.R, ld, k, xb, par, sh, wabs, wval, widx);
    const int jstar = sh.idx;
    const double delta = jstar >= 0 ? sh.val : 0.0;
    if (delta == 0.0) {
      // The row is already represented exactly: move to the best-scored
      // unused row (rows are marked used above).
      ++zero_rows;
#pragma unroll
      for (int s = 0; s < RPT; ++s) cand[s] = ok[s] && used_r[e[s] - row0] == 0;
      __syncthreads();
      cluster_reduce<T, RPT>(cl, CS, score, ok, cand, e, A.C, ld, 0, xb, par, sh, wabs, wval, widx);
      if (zero_rows > A.max_zero_rows || sh.idx < 0) { converged = 1; break; }
      istar = sh.idx;
      continue;
    }
    const double rsq = sh.sumsq;
    for (int l = tid; l < k; l += NT) sh.gr[l] = sh.dots[l] / delta;
    if (jstar >= row0 && jstar < row1 && tid == 0) used_c[jstar - row0] = 1;
    // ---------------- column half-step at jstar
    const T tdelta = (T)delta;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (ok[s]) A.R[e[s] + (size_t)k * ld] = v[s] / tdelta;
    for (int al = tid; al < r; al += NT) s_vec[al] = A.Vh[jstar + (size_t)al * ld];
    for (int l = tid; l < k; l += NT) s_coef[l] = (T)(sh.d[l] * (double)__ldcg(&A.R[jstar + (size_t)l * ld]));
    __syncthreads();
    {
      const T aj = A.a[jstar], bj = A.b[jstar];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        v[s] = T(0);
        if (!ok[s]) continue;
        const int i = e[s];
        T num = T(0);
        for (int al = 0; al < r; ++al) num += A.Uh[i + (size_t)al * ld] * s_vec[al];
        T x = num / (A.a[i] * bj + A.b[i] * aj);
        for (int l = 0; l < k; ++l) x -= A.C[i + (size_t)l * ld] * s_coef[l];
        x = x / tdelta;
        v[s] = x;
        A.C[i + (size_t)k * ld] = x;
        cand[s] = used_r[i - row0] == 0;
      }
    }
    cluster_reduce<T, RPT>(cl, CS, v, ok, cand, e, A.C, ld, k, xb, par, sh, wabs, wval, widx);
    const int inext = sh.idx;
    const double csq = sh.sumsq;
    // ---------------- bookkeeping (identical in every CTA)
    const double rr = rsq / (delta * delta);
    double cross_sum = 0.0;
    if (tid == 0) {
      for (int l = 0; l < k; ++l) cross_sum += sh.d[l] * sh.dots[l] * sh.gr[l];
      sh.d[k] = delta;
    }
    if (q == 0) {
      for (int l = tid; l < k; l += NT) {
        A.GC[l + (size_t)k * A.kcap] = sh.dots[l];
        A.GC[k + (size_t)l * A.kcap] = sh.dots[l];
        A.GR[l + (size_t)k * A.kcap] = sh.gr[l];
        A.GR[k + (size_t)l * A.kcap] = sh.gr[l];
      }
      if (tid == 0) {
        A.GC[k + (size_t)k * A.kcap] = csq;
        A.GR[k + (size_t)k * A.kcap] = rr;
        A.d[k] = delta;
        A.I[k] = istar;
        A.J[k] = jstar;
      }
    }
    if (tid == 0) {
      norm2 += 2.0 * delta * cross_sum + delta * delta * csq * rr;
      sh.val = norm2;
    }
    __syncthreads();
    norm2 = sh.val;
    ++k;
    const double term = fabs(delta) * sqrt(csq * rr);
    small = (term <= A.tol * sqrt(fmax(norm2, 0.0))) ? small + 1 : 0;
    if (small >= 2) {
      if (probe_rounds >= A.max_probe_rounds || A.probes <= 0) { converged = 1; break; }
      // Residual probes at splitmix64-drawn entries; one warp per probe, the
      // same arithmetic in every CTA.
      int P = A.probes < 32 ? A.probes : 32;
      if (P > (NT >> 5)) P = NT >> 5;
      if (warp < P) {
        const unsigned long long z = splitmix64_at(A.seed + (unsigned long long)probe_rounds,
                                                   (unsigned long long)(warp + 1));
        const int pi = (int)((z >> 32) % (unsigned long long)m);
        const int pj = (int)((z & 0xFFFFFFFFULL) % (unsigned long long)m);
        double num = 0.0, sk = 0.0;
        for (int al = lane; al < r; al += 32)
          num += (double)A.Uh[pi + (size_t)al * ld] * (double)A.Vh[pj + (size_t)al * ld];
        for (int l = lane; l < k; l += 32)
          sk += (double)__ldcg(&A.C[pi + (size_t)l * ld]) * sh.d[l] *
                (double)__ldcg(&A.R[pj + (size_t)l * ld]);
        num = warp_sum(num);
        sk = warp_sum(sk);
        const double den = (double)A.a[pi] * (double)A.b[pj] + (double)A.b[pi] * (double)A.a[pj];
        if (lane == 0) { s_probe[warp] = fabs(num / den - sk); s_probe_row[warp] = pi; }
      }
      __syncthreads();
      if (tid == 0) {
        double worst = -1.0;
        int wrow = -1;
        for (int p = 0; p < P; ++p)
          if (s_probe[p] > worst) { worst = s_probe[p]; wrow = s_probe_row[p]; }
        sh.flag = worst <= A.tol * sqrt(fmax(norm2, 0.0)) ? -1 : wrow;
      }
      __syncthreads();
      ++probe_rounds;
      const int bad_row = sh.flag;
      if (bad_row < 0) { converged = 1; break; }
      small = 0;
      // Restart at the bad probe's row if unused, else at the best unused score.
      bool row_used = false;
      if (bad_row >= row0 && bad_row < row1) row_used = used_r[bad_row - row0] != 0;
      // every CTA needs the owner's answer: publish through the score reduction
#pragma unroll
      for (int s = 0; s < RPT; ++s) cand[s] = ok[s] && used_r[e[s] - row0] == 0;
      T bump[RPT];
#pragma unroll
      for (int s = 0; s < RPT; ++s) bump[s] = (ok[s] && e[s] == bad_row && !row_used) ? T(INFINITY) : score[s];
      __syncthreads();
      cluster_reduce<T, RPT>(cl, CS, bump, ok, cand, e, A.C, ld, 0, xb, par, sh, wabs, wval, widx);
      istar = sh.idx;
      if (istar < 0) { converged = 1; break; }
      continue;
    }
    istar = inext;
    if (istar < 0) { converged = 1; break; }
  }
  // No CTA may exit while another can still read its shared memory.
  cl.sync();
  if (q == 0 && tid == 0) {
    A.st->k = k;
    A.st->converged = converged;
    A.st->probe_rounds = probe_rounds;
    A.st->zero_rows = zero_rows;
    A.st->norm2 = norm2;
  }
  (void)lane;
}

template <typename T, int RPT>
static cudaError_t launch_cross_rpt(const CrossArgs<T>& a, int cs, int nt, size_t dsmem, cudaStream_t st) {
  auto kern = cross_kernel<T, RPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
  if (e != cudaSuccess) return e;
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
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T>
cudaError_t launch_cross(const CrossArgs<T>& a, int cluster_size, cudaStream_t st, int* used_cluster) {
  int cs = cluster_size;
  if (cs <= 0) {
    cs = (a.m + 1023) / 1024;
    if (cs > 16) cs = 16;
    if (cs < 1) cs = 1;
  }
  cudaError_t e = cudaErrorInvalidConfiguration;
  for (; cs >= 1; cs = (cs > 8 ? 8 : cs - 1)) {
    const int S = (a.m + cs - 1) / cs;
    int nt = ((S + 31) / 32) * 32;
    if (nt > 1024) nt = 1024;
    if (nt < 64) nt = 64;
    const int rpt = (S + nt - 1) / nt;
    const size_t dsmem = (size_t)((2 * S + 15) / 16) * 16;
    if (rpt <= 1) e = launch_cross_rpt<T, 1>(a, cs, nt, dsmem, st);
    else if (rpt <= 2) e = launch_cross_rpt<T, 2>(a, cs, nt, dsmem, st);
    else if (rpt <= 4) e = launch_cross_rpt<T, 4>(a, cs, nt, dsmem, st);
    else if (rpt <= 8) e = launch_cross_rpt<T, 8>(a, cs, nt, dsmem, st);
    else e = cudaErrorInvalidValue;  // m too large for this cluster size
    if (e == cudaSuccess) { if (used_cluster) *used_cluster = cs; return e; }
    if (e != cudaErrorInvalidConfiguration && e != cudaErrorInvalidValue &&
        e != cudaErrorInvalidClusterSize && e != cudaErrorLaunchOutOfResources)
      return e;
    cudaGetLastError();  // clear the launch-configuration error and retry smaller
  }
  return e;
}

template cudaError_t launch_cross<double>(const CrossArgs<double>&, int, cudaStream_t, int*);
template cudaError_t launch_cross<float>(const CrossArgs<float>&, int, cudaStream_t, int*);

}  // namespace lrp
