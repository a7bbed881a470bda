// Maxvol row selection: the quasi-optimal choice of the cross's rows that
// Section 4.2 cites (Goreinov, Oseledets, Savostyanov, Tyrtyshnikov and
// Zamarashkin, "How to find a good submatrix", 2010).
//
// C is m x k (k <= 64) with k selected rows I.  B = C C[I, :]^{-1} holds the
// coefficients of every row of C in the basis of the rows I (B[I, :] is the
// identity by definition and is stored as such).  While the largest |B[i, j]|
// (lowest column-major index j m + i on ties) exceeds 1 + delta, row i
// replaces I[j] -- which multiplies |det C[I, :]| by |B[i, j]| -- and B takes
// the rank-1 update
//   B' = B - B[:, j] (B[i, :] - e_j^T) / B[i, j]    (row i becomes e_j^T).
//
// Kernels, float64 throughout:
//   mv_inverse  one CTA: Gauss-Jordan inverse of C[I, :] with partial
//               pivoting, [A | identity] held in shared memory (2 k^2 doubles);
//   mv_coeff    grid-stride over rows: B[i, :] = C[i, :] C[I, :]^{-1}, the row of
//               C in registers, the inverse in shared memory;
//   mv_swap     grid-stride over rows: the rank-1 update, one thread per row
//               (it loads the whole row into registers, B[i, j] included,
//               before it rewrites it); row i set to e_j.
// mv_coeff and mv_swap end with the decision: per-CTA argmax of |B| to a
// partial, then the last CTA to finish (a ticket counter: nobody waits)
// reduces the partials, records the next swap or the stop, and copies the
// pivot row B[i, :] for the next update.  The host launches swaps in groups
// of 32 and reads the record between groups; a swap launched after the stop
// returns at once.
#include <cfloat>
#include <climits>

#include "maxvol.h"

namespace lrp {

namespace {

__device__ __forceinline__ bool mv_better(double a_abs, long long a_idx, double b_abs, long long b_idx) {
  return a_abs > b_abs || (a_abs == b_abs && a_idx < b_idx);
}

// Running argmax of |v| on the magnitude bits: for finite doubles the order of
// |v| is the unsigned order of the bit pattern with the sign cleared, so the
// per-element work stays off the (slow) float64 pipe.
__device__ __forceinline__ void mv_track(double v, long long idx, unsigned long long& bbits, long long& bidx,
                                         bool& nonfinite) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
  if (a >= 0x7FF0000000000000ULL) nonfinite = true;
  else if (a > bbits || (a == bbits && idx < bidx)) { bbits = a; bidx = idx; }
}

__device__ __forceinline__ void mv_warp_best(double& babs, long long& bidx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double oa = __shfl_xor_sync(0xffffffffu, babs, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (mv_better(oa, oi, babs, bidx)) { babs = oa; bidx = oi; }
  }
}

// Largest (|B|, index) over the CTA, valid in thread 0.
__device__ void mv_block_best(double& babs, long long& bidx) {
  __shared__ double sa[MV_THREADS / 32];
  __shared__ long long si[MV_THREADS / 32];
  mv_warp_best(babs, bidx);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sa[w] = babs; si[w] = bidx; }
  __syncthreads();
  if (w == 0) {
    babs = lane < MV_THREADS / 32 ? sa[lane] : -1.0;
    bidx = lane < MV_THREADS / 32 ? si[lane] : LLONG_MAX;
    mv_warp_best(babs, bidx);
  }
  __syncthreads();
}

// The decision after B has been written: CTA partial, then the last CTA
// reduces all partials and records the next swap or the stop.  A thread that
// saw no finite entry holds bbits = 0 with bidx = LLONG_MAX, which any real
// entry beats.
__device__ void mv_decide(const MvArgs& a, unsigned long long bbits, long long bidx, bool nonfinite) {
  __shared__ int s_last, s_go, s_i;
  double babs = bidx == LLONG_MAX ? -1.0 : __longlong_as_double((long long)bbits);
  const bool bad = __syncthreads_or(nonfinite ? 1 : 0) != 0;
  mv_block_best(babs, bidx);
  if (threadIdx.x == 0) {
    a.pabs[blockIdx.x] = babs;
    a.pidx[blockIdx.x] = bidx;
    if (bad) atomicOr(&a.st->status, 2);
    __threadfence();
    const unsigned t = atomicAdd(&a.st->ticket, 1u);
    s_last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  babs = -1.0;
  bidx = LLONG_MAX;
  for (int g = threadIdx.x; g < (int)gridDim.x; g += blockDim.x) {
    const double v = __ldcg(a.pabs + g);
    const long long ix = __ldcg(a.pidx + g);
    if (mv_better(v, ix, babs, bidx)) { babs = v; bidx = ix; }
  }
  mv_block_best(babs, bidx);
  if (threadIdx.x == 0) {
    MvState* s = a.st;
    s->ticket = 0;
    const int status = atomicOr(&s->status, 0);
    const int nsw = __ldcg(&s->nswaps);
    s->bmax = babs;
    int go = 0;
    if (status == 0 && babs > 1.0 + a.delta && nsw < a.maxswaps) {
      const int i = (int)(bidx % a.m), j = (int)(bidx / a.m);
      s->i = i;
      s->j = j;
      s->piv = __ldcg(a.B + i + (size_t)j * a.ldb);
      a.rows[j] = i;
      s->nswaps = nsw + 1;
      s_i = i;
      go = 1;
    } else {
      s->done = 1;
    }
    s_go = go;
  }
  __syncthreads();
  if (s_go)
    for (int l = threadIdx.x; l < a.k; l += blockDim.x) a.row[l] = __ldcg(a.B + s_i + (size_t)l * a.ldb);
}

__global__ void __launch_bounds__(MV_THREADS) mv_inverse_kernel(MvArgs a) {
  extern __shared__ double M[];  // k rows of 2k: [A | identity] -> [identity | A^{-1}]
  __shared__ double fac[MV_KMAX];
  __shared__ int s_p, s_bad;
  const int k = a.k, w = 2 * k;
  for (int x = threadIdx.x; x < k * w; x += blockDim.x) {
    const int r = x / w, c = x - r * w;
    M[x] = c < k ? a.C[(size_t)a.rows[r] + (size_t)c * a.ldc] : (c - k == r ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double bv = fabs(M[c * w + c]);
      for (int r = c + 1; r < k; ++r) {
        const double v = fabs(M[r * w + c]);
        if (v > bv) { bv = v; p = r; }
      }
      s_p = p;
      s_bad = !(bv > 0.0 && bv <= DBL_MAX);
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_p;
    if (p != c)
      for (int x = threadIdx.x; x < w; x += blockDim.x) {
        const double t = M[c * w + x];
        M[c * w + x] = M[p * w + x];
        M[p * w + x] = t;
      }
    __syncthreads();
    const double inv = 1.0 / M[c * w + c];
    __syncthreads();
    for (int x = threadIdx.x; x < w; x += blockDim.x) M[c * w + x] *= inv;
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x) fac[r] = M[r * w + c];
    __syncthreads();
    for (int x = threadIdx.x; x < k * w; x += blockDim.x) {
      const int r = x / w, y = x - r * w;
      if (r != c) M[x] -= fac[r] * M[c * w + y];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(&a.st->status, 1);
      a.st->done = 1;
    }
    return;
  }
  for (int x = threadIdx.x; x < MV_KMAX * MV_KMAX; x += blockDim.x) {
    const int p = x / MV_KMAX, l = x - p * MV_KMAX;
    a.Ainv[x] = (p < k && l < k) ? M[p * w + k + l] : 0.0;
  }
}

template <int KC>
__global__ void __launch_bounds__(MV_THREADS) mv_coeff_kernel(MvArgs a) {
  __shared__ double Ai[KC * KC];
  __shared__ int srow[MV_KMAX];
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = __ldcg(&a.st->done);
  for (int x = threadIdx.x; x < KC * KC; x += blockDim.x) Ai[x] = a.Ainv[(x / KC) * MV_KMAX + (x % KC)];
  for (int j = threadIdx.x; j < a.k; j += blockDim.x) srow[j] = a.rows[j];
  __syncthreads();
  if (s_done) return;
  const int k = a.k, m = a.m;
  unsigned long long bbits = 0;
  long long bidx = LLONG_MAX;
  bool nonfinite = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double* bi = a.B + i;
    int sel = -1;
    for (int j = 0; j < k; ++j)
      if (srow[j] == i) sel = j;
    if (sel >= 0) {
      for (int l = 0; l < k; ++l) {
        const double v = l == sel ? 1.0 : 0.0;
        bi[(size_t)l * a.ldb] = v;
        mv_track(v, (long long)l * m + i, bbits, bidx, nonfinite);
      }
      continue;
    }
    double cr[KC];
#pragma unroll
    for (int p = 0; p < KC; ++p) cr[p] = p < k ? a.C[(size_t)i + (size_t)p * a.ldc] : 0.0;
    for (int l = 0; l < k; ++l) {
      double acc = 0.0;
#pragma unroll
      for (int p = 0; p < KC; ++p) acc = fma(cr[p], Ai[p * KC + l], acc);
      bi[(size_t)l * a.ldb] = acc;
      mv_track(acc, (long long)l * m + i, bbits, bidx, nonfinite);
    }
  }
  mv_decide(a, bbits, bidx, nonfinite);
}

template <int KC>
__global__ void __launch_bounds__(MV_THREADS) mv_swap_kernel(MvArgs a) {
  __shared__ double r[MV_KMAX];
  __shared__ int s_done, s_i, s_j;
  __shared__ double s_piv;
  if (threadIdx.x == 0) {
    s_done = __ldcg(&a.st->done);
    s_i = __ldcg(&a.st->i);
    s_j = __ldcg(&a.st->j);
    s_piv = __ldcg(&a.st->piv);
  }
  __syncthreads();
  if (s_done) return;
  const int k = a.k, m = a.m, is = s_i, js = s_j;
  const double piv = s_piv;
  for (int l = threadIdx.x; l < k; l += blockDim.x) r[l] = __ldcg(a.row + l) - (l == js ? 1.0 : 0.0);
  __syncthreads();
  unsigned long long bbits = 0;
  long long bidx = LLONG_MAX;
  bool nonfinite = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double* bi = a.B + i;
    if (i == is) {
      for (int l = 0; l < k; ++l) {
        const double v = l == js ? 1.0 : 0.0;
        bi[(size_t)l * a.ldb] = v;
        mv_track(v, (long long)l * m + i, bbits, bidx, nonfinite);
      }
    } else {
      double b[KC];
#pragma unroll
      for (int l = 0; l < KC; ++l)
        if (l < k) b[l] = bi[(size_t)l * a.ldb];
      const double f = bi[(size_t)js * a.ldb] / piv;
#pragma unroll
      for (int l = 0; l < KC; ++l)
        if (l < k) {
          const double v = fma(-f, r[l], b[l]);
          bi[(size_t)l * a.ldb] = v;
          mv_track(v, (long long)l * m + i, bbits, bidx, nonfinite);
        }
    }
  }
  mv_decide(a, bbits, bidx, nonfinite);
}

}  // namespace

int maxvol_grid(int m, int num_sms) {
  const int need = (m + MV_THREADS - 1) / MV_THREADS;
  const int cap = 2 * (num_sms > 0 ? num_sms : 1);
  return need < cap ? (need > 0 ? need : 1) : cap;
}

cudaError_t launch_maxvol_start(const MvArgs& a, cudaStream_t st) {
  if (a.k < 1 || a.k > MV_KMAX || a.m < a.k || a.grid < 1) return cudaErrorInvalidValue;
  const int smem = 2 * a.k * a.k * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(mv_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * MV_KMAX * MV_KMAX * (int)sizeof(double));
  if (e != cudaSuccess) return e;
  mv_inverse_kernel<<<1, MV_THREADS, smem, st>>>(a);
  if (a.k <= 8) mv_coeff_kernel<8><<<a.grid, MV_THREADS, 0, st>>>(a);
  else if (a.k <= 16) mv_coeff_kernel<16><<<a.grid, MV_THREADS, 0, st>>>(a);
  else if (a.k <= 32) mv_coeff_kernel<32><<<a.grid, MV_THREADS, 0, st>>>(a);
  else mv_coeff_kernel<64><<<a.grid, MV_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_maxvol_swap(const MvArgs& a, cudaStream_t st) {
  if (a.k < 1 || a.k > MV_KMAX || a.grid < 1) return cudaErrorInvalidValue;
  if (a.k <= 8) mv_swap_kernel<8><<<a.grid, MV_THREADS, 0, st>>>(a);
  else if (a.k <= 16) mv_swap_kernel<16><<<a.grid, MV_THREADS, 0, st>>>(a);
  else if (a.k <= 32) mv_swap_kernel<32><<<a.grid, MV_THREADS, 0, st>>>(a);
  else mv_swap_kernel<64><<<a.grid, MV_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lrp
