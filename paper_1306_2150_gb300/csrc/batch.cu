// Phase-batched low-rank solves: the steps of the Section 4.2 solve (forward
// DST of the factors, cross in frequency space, rounding, inverse DST) for
// every problem of a batch, one launch per step instead of one launch chain
// per problem.
//
// Problems are described on the device (BatchProb).  A launch walks a flat
// item space; an item finds its problem by binary search in the launch's
// prefix table, so problems of different order and rank share one grid.
//
// Transforms (Section 4.1, Eq. flr:diag): the Bluestein evaluation of dst.cu
// (chirp, power-of-two FFT of length M >= 2m - 1, kernel spectrum, inverse
// FFT, chirp), with tiles of 4096 complex elements:
//   M <= 4096 : one item = 4096 / M columns of one problem, whole sequences in
//               shared memory;
//   M >  4096 : four-step split M = M1 M2 through the problem's global scratch
//               (column pass, row pass with the spectrum product, column pass).
// All shared-memory FFT lengths are at most 4096, so every CTA builds the
// stage twiddle tables (fft_common.cuh) once, from one table of length 4096.
//
// Cross (Section 4.2, Eq. flr:div): one CTA, or a cluster of 2 or 4 CTAs, per
// problem.  A CTA owns a contiguous slice of indices; thread t owns indices
// row0 + t + s NT (s < RPT), so every column access of a warp is one
// coalesced 128-byte line.  Factors and skeleton are read from global memory
// (L2): the CTA's shared memory holds only reduction partials, so several
// problems' CTAs can share an SM.  A half-step: evaluate the owned residual
// entries, warp reductions (argmax with lowest index on ties, sum of squares,
// dot products with the skeleton columns for the Gram matrices), each warp
// fetches the pivot data its own candidate would need next, one CTA
// reduction; in a cluster the CTA partials are pushed into every CTA's inbox
// (distributed shared memory) and reduced in rank order after one cluster
// barrier, so all CTAs take the same decision with the same arithmetic.  The
// decisions (pivots, zero rows, stop rule, residual probes, restarts) are
// those of the single-solve cross kernel (cross.cu) and of the oracle.
#include <cooperative_groups.h>

#include <climits>

#include "fft_common.cuh"
#include "lr_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

namespace {

__device__ __forceinline__ int find_item(const int* __restrict__ start, int n, int item) {
  // largest q with start[q] <= item (start[0] = 0, start[n] = total)
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&start[mid]) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Column addressing of a batched transform.  dir 0: column c < 2r of
// [U V] -> [Uh Vh]; dir 1: column c < 2 ncap of W -> [Uo Vo], live while its
// index within its factor is below the kept rank.
template <typename T, int DIR>
struct BCol {
  const void* in;
  void* out;
  bool live;
  __device__ __forceinline__ BCol(const BatchProb& B, int col) {
    if (DIR == 0) {
      const int seg = col < B.r ? 0 : 1, cc = col - seg * B.r;
      live = col < 2 * B.r;
      in = (seg ? B.V : B.U) + (size_t)cc * B.ld_in;
      out = static_cast<T*>(seg ? B.Vh : B.Uh) + (size_t)cc * B.ldw;
    } else {
      const int seg = col < B.ncap ? 0 : 1, cc = col - seg * B.ncap;
      live = col < 2 * B.ncap && cc < B.st->rank;
      in = static_cast<const T*>(B.W) + (size_t)col * B.ldw;
      out = (seg ? B.Vo : B.Uo) + (size_t)cc * B.ld_out;
    }
  }
  __device__ __forceinline__ T load(int t) const {
    if (DIR == 0) return (T)static_cast<const double*>(in)[t];
    return static_cast<const T*>(in)[t];
  }
  __device__ __forceinline__ void store(int t, T v) const {
    if (DIR == 0) static_cast<T*>(out)[t] = v;
    else static_cast<double*>(out)[t] = (double)v;
  }
};

// Column of the inverse transform for dense live index c (0 <= c < 2R:
// U columns 0..R-1, then V columns ncap..ncap+R-1), -1 past the live ones.
__device__ __forceinline__ int live_col(const BatchProb& B, int c) {
  const int R = B.st->rank;
  return c < R ? c : (c < 2 * R ? B.ncap + (c - R) : -1);
}

// Items of a launch: fixed, or counted on the device (live columns).
__device__ __forceinline__ int item_count(const BatchItems& it) {
  return it.live ? __ldcg(&it.start[it.n]) : it.items;
}
__device__ __forceinline__ int find_live_item(const BatchItems& it, int item) {
  // as find_item, over a table written by an earlier launch (no read-only path)
  int lo = 0, hi = it.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldcg(&it.start[mid]) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kBTile = 4096;          // complex elements per tile
constexpr int kBThreads = kBTile / EPT;


// ---- M <= 4096: whole sequences in shared memory ---------------------------
template <typename T, int DIR>
__global__ void __launch_bounds__(kBThreads, 2) bdst_small_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                               const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);  // padded tile (smem_ix<true>)
  cpx<T>* stw = buf + kBTile + (kBTile >> 4);
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  const int items = item_count(it);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
    const BatchProb& B = P[it.list[q]];
    const int logM = B.logM, M = 1 << logM, lognf = 12 - logM;
    const int col0 = (item - __ldcg(&it.start[q])) << lognf;
    const cpx<T>* chirp = static_cast<const cpx<T>*>(B.chirp);
    const cpx<T>* bhat = static_cast<const cpx<T>*>(B.bhat);
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        const int t = idx & (M - 1);
        const int cl = it.live ? live_col(B, col0 + (idx >> logM)) : col0 + (idx >> logM);
        const BCol<T, DIR> c(B, cl < 0 ? 2 * B.ncap : cl);
        v[s] = {T(0), T(0)};
        if (c.live && t < B.m) {
          const T x = c.load(t);
          const cpx<T> w = chirp[t];
          v[s] = {x * w.re, x * w.im};
        }
      }
      __syncthreads();  // the previous item's stores read buf
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[smem_ix<true>(threadIdx.x + s * kBThreads)] = v[s];
    }
    __syncthreads();
    smem_fft_st<T, false, true>(buf, logM, lognf, 1, M, stw, stride, false);
    {
      cpx<T> b[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) b[s] = bhat[(threadIdx.x + s * kBThreads) & (M - 1)];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = smem_ix<true>(threadIdx.x + s * kBThreads);
        buf[idx] = cmul(buf[idx], b[s]);
      }
    }
    __syncthreads();
    smem_fft_st<T, false, true>(buf, logM, lognf, 1, M, stw, stride, true);
#pragma unroll
    for (int s = 0; s < EPT; ++s) {
      const int idx = threadIdx.x + s * kBThreads;
      const int t = idx & (M - 1);
      const int cl = it.live ? live_col(B, col0 + (idx >> logM)) : col0 + (idx >> logM);
      const BCol<T, DIR> c(B, cl < 0 ? 2 * B.ncap : cl);
      if (c.live && t < B.m) {
        const cpx<T> w = chirp[t], z = buf[smem_ix<true>(idx)];
        c.store(t, w.re * z.im + w.im * z.re);  // Im(w z)
      }
    }
  }
}

// ---- M > 4096, four-step: index t = t1 + M1 t2, frequency k = k2 + M2 k1,
// scratch of each column stored as [k2][t1] (see dst.cu).  Column passes:
// a tile holds TX = 4096 / M2 consecutive t1 and all M2 values of t2 (k2).
template <typename T, int DIR>
__global__ void __launch_bounds__(kBThreads, 2) bdst_col_fwd_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                                 const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* stw = buf + kBTile + 512;  // after the (row pass: padded) tile
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  cpx<T>* th = stw + stage_elems<T>(it.slog);  // inter-pass twiddles of the current M
  cpx<T>* tl = th + kTwHi;
  int curM = 0;
  const int items = item_count(it);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2;
    const int logTX = 12 - logM2, TX = 1 << logTX;
    const int bpc = (1 << logM1) >> logTX;
    const int local = item - __ldcg(&it.start[q]);
    const int lc = local / bpc;
    const int col = it.live ? live_col(B, lc) : lc;
    const int t1_0 = (local - lc * bpc) << logTX;
    const BCol<T, DIR> c(B, col < 0 ? 2 * B.ncap : col);
    if (!c.live) continue;  // uniform across the CTA
    const cpx<T>* chirp = static_cast<const cpx<T>*>(B.chirp);
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        const int t = t1_0 + (idx & (TX - 1)) + ((idx >> logTX) << logM1);
        v[s] = {T(0), T(0)};
        if (t < B.m) {
          const T x = c.load(t);
          const cpx<T> w = chirp[t];
          v[s] = {x * w.re, x * w.im};
        }
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[threadIdx.x + s * kBThreads] = v[s];
      if (B.logM != curM) {  // uniform across the CTA
        load_twiddles2(th, tl, static_cast<const cpx<T>*>(B.tw), B.logM);
        curM = B.logM;
      }
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, logM2, logTX, TX, 1, stw, stride, false);
    cpx<T>* wc = static_cast<cpx<T>*>(B.work) + ((size_t)col << B.logM);
    {
      cpx<T> w[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        w[s] = twiddle2(th, tl, (t1_0 + (idx & (TX - 1))) * (idx >> logTX));
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        wc[((idx >> logTX) << logM1) + t1_0 + (idx & (TX - 1))] = cmul(buf[idx], w[s]);
      }
    }
  }
}

// Row pass: RY = 4096 / M1 rows k2 per tile, each of M1 contiguous elements.
template <typename T, int DIR>
__global__ void __launch_bounds__(kBThreads, 2) bdst_row_mid_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                                 const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* stw = buf + kBTile + 512;  // after the (row pass: padded) tile
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  cpx<T>* th = stw + stage_elems<T>(it.slog);  // inter-pass twiddles of the current M
  cpx<T>* tl = th + kTwHi;
  int curM = 0;
  const int items = item_count(it);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2, M1 = 1 << logM1;
    const int logRY = 12 - logM1;
    const int bpc = (1 << logM2) >> logRY;
    const int local = item - __ldcg(&it.start[q]);
    const int lc = local / bpc;
    const int col = it.live ? live_col(B, lc) : lc;
    const int k2_0 = (local - lc * bpc) << logRY;
    const BCol<T, DIR> c(B, col < 0 ? 2 * B.ncap : col);
    if (!c.live) continue;
    cpx<T>* wc = static_cast<cpx<T>*>(B.work) + ((size_t)col << B.logM) + ((size_t)k2_0 << logM1);
    const cpx<T>* bh = static_cast<const cpx<T>*>(B.bhat) + ((size_t)k2_0 << logM1);
    // rows interleaved in shared memory (element e of row f at e (RY + 1) + f):
    // the FFT passes then run with consecutive lanes on consecutive rows
    const int ES = (1 << logRY) + 1;
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) v[s] = wc[threadIdx.x + s * kBThreads];
      __syncthreads();
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        buf[(idx & (M1 - 1)) * ES + (idx >> logM1)] = v[s];
      }
      if (B.logM != curM) {  // uniform across the CTA
        load_twiddles2(th, tl, static_cast<const cpx<T>*>(B.tw), B.logM);
        curM = B.logM;
      }
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, logM1, logRY, ES, 1, stw, stride, false);
    {
      cpx<T> b[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) b[s] = bh[threadIdx.x + s * kBThreads];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        const int bi = (idx & (M1 - 1)) * ES + (idx >> logM1);
        buf[bi] = cmul(buf[bi], b[s]);
      }
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, logM1, logRY, ES, 1, stw, stride, true);
    {
      cpx<T> w[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        w[s] = twiddle2(th, tl, (idx & (M1 - 1)) * (k2_0 + (idx >> logM1)));
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        wc[idx] = cmulc(buf[(idx & (M1 - 1)) * ES + (idx >> logM1)], w[s]);  // times exp(+2 pi i t1 k2 / M)
      }
    }
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(kBThreads, 2) bdst_col_inv_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                                 const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* stw = buf + kBTile + 512;  // after the (row pass: padded) tile
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  const int items = item_count(it);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2;
    const int logTX = 12 - logM2, TX = 1 << logTX;
    const int bpc = (1 << logM1) >> logTX;
    const int local = item - __ldcg(&it.start[q]);
    const int lc = local / bpc;
    const int col = it.live ? live_col(B, lc) : lc;
    const int t1_0 = (local - lc * bpc) << logTX;
    const BCol<T, DIR> c(B, col < 0 ? 2 * B.ncap : col);
    if (!c.live) continue;
    const cpx<T>* chirp = static_cast<const cpx<T>*>(B.chirp);
    const cpx<T>* wc = static_cast<const cpx<T>*>(B.work) + ((size_t)col << B.logM);
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * kBThreads;
        v[s] = wc[((idx >> logTX) << logM1) + t1_0 + (idx & (TX - 1))];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[threadIdx.x + s * kBThreads] = v[s];
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, logM2, logTX, TX, 1, stw, stride, true);
#pragma unroll
    for (int s = 0; s < EPT; ++s) {
      const int idx = threadIdx.x + s * kBThreads;
      const int t = t1_0 + (idx & (TX - 1)) + ((idx >> logTX) << logM1);
      if (t < B.m) {
        const cpx<T> w = chirp[t], z = buf[idx];
        c.store(t, w.re * z.im + w.im * z.re);
      }
    }
  }
}

template <typename T, int DIR>
cudaError_t launch_bdst_dir(const BatchProb* probs, const BatchItems& small, const BatchItems& col,
                            const BatchItems& row, const cpx<T>* tw, int num_sms, cudaStream_t st) {
  // tile (padded by 1/16, or by up to 512 for the row pass) + stage tables
  // tile (padded by 1/16, or by up to 512 for the row pass), stage tables,
  // inter-pass twiddles
  const size_t smax = ((size_t)kBTile + 512 + stage_elems<T>(kStageLog) + kTwHi + kTwLo) * sizeof(cpx<T>);
  auto bytes = [](const BatchItems& b) {
    return ((size_t)kBTile + 512 + stage_elems<T>(b.slog) + kTwHi + kTwLo) * sizeof(cpx<T>);
  };
  auto k0 = bdst_small_kernel<T, DIR>;
  auto k1 = bdst_col_fwd_kernel<T, DIR>;
  auto k2 = bdst_row_mid_kernel<T, DIR>;
  auto k3 = bdst_col_inv_kernel<T, DIR>;
  static cudaError_t attr = [&] {
    cudaError_t e = cudaSuccess;
    for (const void* k : {(const void*)k0, (const void*)k1, (const void*)k2, (const void*)k3}) {
      cudaError_t ek = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
      if (ek == cudaSuccess)  // let several CTAs share an SM's shared memory
        ek = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (ek != cudaSuccess) e = ek;
    }
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  // grid: enough CTAs for every item, at most 4 per SM (grid-stride beyond)
  const int cap = 4 * num_sms;
  if (small.items > 0) k0<<<small.items < cap ? small.items : cap, kBThreads, bytes(small), st>>>(probs, small, tw);
  if (col.items > 0) {
    k1<<<col.items < cap ? col.items : cap, kBThreads, bytes(col), st>>>(probs, col, tw);
    k2<<<row.items < cap ? row.items : cap, kBThreads, bytes(row), st>>>(probs, row, tw);
    k3<<<col.items < cap ? col.items : cap, kBThreads, bytes(col), st>>>(probs, col, tw);
  }
  return cudaGetLastError();
}

// Exclusive scan of per-problem live item counts into start[0..n] (one CTA).
__device__ void live_scan(const BatchProb* __restrict__ P, const BatchItems& it, int kind) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
  int* start = const_cast<int*>(it.start);
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < it.n; base += blockDim.x) {
    const int q = base + tid;
    int cnt = 0;
    if (q < it.n) {
      const BatchProb& B = P[it.list[q]];
      const int cols = 2 * B.st->rank;
      if (kind == 0) {
        const int nf = 1 << (12 - B.logM);
        cnt = (cols + nf - 1) / nf;
      } else if (kind == 1) {
        cnt = cols * ((1 << B.logM1) >> (12 - B.logM2));
      } else {
        cnt = cols * ((1 << B.logM2) >> (12 - B.logM1));
      }
    }
    int x = cnt;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < NW ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < NW) wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int before = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - cnt;
    if (q < it.n) start[q] = before;
    __syncthreads();
    if (tid == 0) carry += wsum[NW - 1];
    __syncthreads();
  }
  if (tid == 0) start[it.n] = carry;
  __syncthreads();
}

__global__ void __launch_bounds__(1024) blive_items_kernel(const BatchProb* __restrict__ P, BatchItems small,
                                                           BatchItems col, BatchItems row) {
  if (small.n > 0) live_scan(P, small, 0);
  if (col.n > 0) live_scan(P, col, 1);
  if (row.n > 0) live_scan(P, row, 2);
}

}  // namespace

cudaError_t launch_batch_live_items(const BatchProb* probs, const BatchItems& small, const BatchItems& col,
                                    const BatchItems& row, cudaStream_t st) {
  if (small.n + col.n + row.n == 0) return cudaSuccess;
  blive_items_kernel<<<1, 1024, 0, st>>>(probs, small, col, row);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_dst(const BatchProb* probs, int dir, const BatchItems& small, const BatchItems& col,
                             const BatchItems& row, const void* tw4096, int num_sms, cudaStream_t st) {
  const cpx<T>* tw = static_cast<const cpx<T>*>(tw4096);
  return dir == 0 ? launch_bdst_dir<T, 0>(probs, small, col, row, tw, num_sms, st)
                  : launch_bdst_dir<T, 1>(probs, small, col, row, tw, num_sms, st);
}
template cudaError_t launch_batch_dst<float>(const BatchProb*, int, const BatchItems&, const BatchItems&,
                                             const BatchItems&, const void*, int, cudaStream_t);
template cudaError_t launch_batch_dst<double>(const BatchProb*, int, const BatchItems&, const BatchItems&,
                                              const BatchItems&, const void*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Rotation W[:, q] = C Tc[:, q], W[:, ncap + q] = R Tr[:, q] (q < rank): the
// last step of the rounding (Section 3), before the inverse transform.  One
// thread per row, both factors; Tc and Tr staged in shared memory per item.
// ---------------------------------------------------------------------------
namespace {
template <typename T>
__global__ void __launch_bounds__(256) brotate_kernel(const BatchProb* __restrict__ P, BatchItems it) {
  extern __shared__ __align__(16) unsigned char rot_raw[];
  T (*tm)[KMAX * KMAX] = reinterpret_cast<T (*)[KMAX * KMAX]>(rot_raw);  // [2][KMAX * KMAX]
  const int items = item_count(it);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
    const BatchProb& B = P[it.list[q]];
    const int k = B.st->k, R = B.st->rank;
    __syncthreads();  // the previous item's rows read tm
    if (R <= 0 || k <= 0) continue;  // uniform across the CTA
    for (int idx = threadIdx.x; idx < k * R; idx += blockDim.x) {
      const int l = idx % k, qq = idx / k;
      tm[0][l + qq * KMAX] = static_cast<const T*>(B.Tc)[l + (size_t)qq * KMAX];
      tm[1][l + qq * KMAX] = static_cast<const T*>(B.Tr)[l + (size_t)qq * KMAX];
    }
    __syncthreads();
    const int row = ((item - it.start[q]) << 8) + threadIdx.x;
    if (row >= B.m) continue;
    for (int side = 0; side < 2; ++side) {
      const T* X = static_cast<const T*>(side ? B.R : B.C) + row;
      T* out = static_cast<T*>(B.W) + (size_t)side * B.ncap * B.ldw + row;
      for (int q0 = 0; q0 < R; q0 += 16) {  // one pass over X for ranks up to 16
        T acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = T(0);
#pragma unroll 4
        for (int l = 0; l < k; ++l) {
          const T x = X[(size_t)l * B.ldw];
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[c] += x * tm[side][l + (q0 + c) * KMAX];
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (q0 + c < R) out[(size_t)(q0 + c) * B.ldw] = acc[c];
      }
    }
  }
}
}  // namespace

template <typename T>
cudaError_t launch_batch_rotate(const BatchProb* probs, const BatchItems& rows, int num_sms, cudaStream_t st) {
  if (rows.items <= 0) return cudaSuccess;
  const int cap = 8 * num_sms;
  const size_t smem = 2 * (size_t)KMAX * KMAX * sizeof(T);
  static cudaError_t attr = cudaFuncSetAttribute(brotate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
  if (attr != cudaSuccess) return attr;
  brotate_kernel<T><<<rows.items < cap ? rows.items : cap, 256, smem, st>>>(probs, rows);
  return cudaGetLastError();
}
template cudaError_t launch_batch_rotate<float>(const BatchProb*, const BatchItems&, int, cudaStream_t);
template cudaError_t launch_batch_rotate<double>(const BatchProb*, const BatchItems&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Batched cross.
// ---------------------------------------------------------------------------
namespace {

constexpr int BX_NT = 512;            // threads per CTA
constexpr int BX_NW = BX_NT / 32;
constexpr int BX_CAND = 2 * KMAX + 3; // candidate pivot data: F row, X row (KMAX + 1), a, b

__device__ __forceinline__ unsigned long long bx_splitmix64_at(unsigned long long state, unsigned long long t) {
  unsigned long long z = state + t * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ bool bx_better(T a_abs, int a_idx, T b_abs, int b_idx) {
  return a_abs > b_abs || (a_abs == b_abs && a_idx < b_idx);
}

template <typename T>
__device__ __forceinline__ T bx_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ void bx_warp_argmax(T& a, int& i, T& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T oa = __shfl_xor_sync(0xffffffffu, a, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    if (bx_better(oa, oi, a, i)) { a = oa; i = oi; v = ov; }
  }
}

template <typename T> __device__ __forceinline__ T bx_ratio(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float bx_ratio<float>(float a, float b) { return __fdividef(a, b); }

// Sum over the warp of a[i], i < 16, for every i at once (recursive halving);
// afterwards lane L holds the sum for index L mod 16.  The addition pattern is
// fixed, so every CTA gets the same bits.
template <typename T>
__device__ __forceinline__ T bx_transpose_sum16(T (&a)[16], int lane) {
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? a[i] : a[i + h];
      const T keep = up ? a[i + h] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 16);
}

// Message of one CTA in a cluster reduction (values of type T): header
// (abs, val, ssq, idx), dot products, candidate pivot data.
template <typename T>
struct BxMsg {
  static constexpr int ABS = 0, VAL = 1, SSQ = 2, IDX = 3, DOTS = 4, CAND = DOTS + KMAX;
  static constexpr int WORDS = CAND + BX_CAND;
};

template <typename T>
struct BxShared {
  T wabs[BX_NW], wval[BX_NW], wsum[BX_NW];
  int widx[BX_NW];
  T wdots[KMAX][BX_NW];
  T wcand[BX_NW][BX_CAND];          // per warp: its candidate's F row, X row, a, b
  T d[KMAX + 1];                    // pivot values
  T dots[KMAX];                     // reduced dot products of the last reduction
  T gr[KMAX];                       // R_l . r of the current step
  T vec[KMAX];                      // pivot row of F for the next half-step
  T cd[KMAX + 1];                   // pivot row of X times d for the next half-step
  T craw[KMAX + 1];                 // pivot row of X
  T piv_a, piv_b;
  double probe[32];
  int probe_row[32];
  T val, sumsq, norm2, rsq, delta, pfloor;
  int idx, win, flag, small;
};

// Problem-level constants of one CTA.  The CTA's slices (local index li =
// j - row0 < SP) of the symbol, of Uh and Vh (if uv) and of the first KS
// skeleton columns live in dynamic shared memory, column-major with leading
// dimension SP; the rest is read from global memory (L2).
template <typename T>
struct BxProb {
  int m, r, ld, kcap, row0, row1;
  const T* Uh;
  const T* Vh;
  T* C;
  T* R;
  const T* a;
  const T* b;
  int SP, KS, uv;
  const T* as;   // symbol slices
  const T* bs;
  const T* Us;   // Uh, Vh slices (uv)
  const T* Vs;
  T* Cs;         // skeleton columns < KS
  T* Rs;
  T* inbox;      // [2][cs][BxMsg::WORDS] cluster partials (dynamic shared memory)
};

// A tall factor as seen by the CTA: global copy, shared copy of columns < ns.
template <typename T>
struct BxSrc {
  const T* g;
  const T* s;
  int ns;
};
template <typename T>
__device__ __forceinline__ T bx_at(const BxProb<T>& p, const BxSrc<T>& S, int l, int li) {
  return l < S.ns ? S.s[(size_t)l * p.SP + li] : __ldcg(&S.g[p.row0 + li + (size_t)l * p.ld]);
}

// out[s] = (vec . F[j]) / (pa b_j + pb a_j) - sum_{l<k} cd[l] X[j, l] for the
// owned indices j = row0 + tid + s NT (0 elsewhere).
template <typename T, int RPT>
__device__ __forceinline__ void bx_eval(const BxProb<T>& p, const BxSrc<T>& F, const BxSrc<T>& X, int k,
                                        const BxShared<T>& sh, T (&out)[RPT]) {
  const int S = p.row1 - p.row0;
  const int tid = threadIdx.x;
#pragma unroll
  for (int s = 0; s < RPT; ++s) out[s] = T(0);
  // F . vec: shared columns, then global ones (uniform loop bounds)
  const int nF = F.ns < p.r ? F.ns : p.r;
#pragma unroll 4
  for (int al = 0; al < nF; ++al) {
    const T w = sh.vec[al];
    const T* Fc = F.s + (size_t)al * p.SP + tid;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (tid + s * BX_NT < S) out[s] += w * Fc[s * BX_NT];
  }
#pragma unroll 4
  for (int al = nF; al < p.r; ++al) {
    const T w = sh.vec[al];
    const T* Fc = F.g + (size_t)al * p.ld + p.row0 + tid;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (tid + s * BX_NT < S) out[s] += w * Fc[s * BX_NT];
  }
  const T pa = sh.piv_a, pb = sh.piv_b;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int li = tid + s * BX_NT;
    out[s] = li < S ? bx_ratio<T>(out[s], pa * p.bs[li] + pb * p.as[li]) : T(0);
  }
  const int nX = X.ns < k ? X.ns : k;
#pragma unroll 4
  for (int l = 0; l < nX; ++l) {
    const T c = sh.cd[l];
    const T* Xc = X.s + (size_t)l * p.SP + tid;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (tid + s * BX_NT < S) out[s] -= c * Xc[s * BX_NT];
  }
#pragma unroll 4
  for (int l = nX; l < k; ++l) {
    const T c = sh.cd[l];
    const T* Xc = X.g + (size_t)l * p.ld + p.row0 + tid;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (tid + s * BX_NT < S) out[s] -= c * __ldcg(&Xc[s * BX_NT]);
  }
}

// Start score ||Uh[j]||^2 / Lambda[j, 0]^2 of the owned indices.
template <typename T, int RPT>
__device__ __forceinline__ void bx_scores(const BxProb<T>& p, T a0, T b0, T (&out)[RPT]) {
  const int S = p.row1 - p.row0;
  const BxSrc<T> U{p.Uh, p.Us, p.uv ? p.r : 0};
#pragma unroll
  for (int s = 0; s < RPT; ++s) out[s] = T(0);
#pragma unroll 4
  for (int al = 0; al < p.r; ++al) {
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int li = threadIdx.x + s * BX_NT;
      if (li < S) { const T u = bx_at(p, U, al, li); out[s] += u * u; }
    }
  }
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int li = threadIdx.x + s * BX_NT;
    if (li < S) {
      const T lam0 = p.as[li] * b0 + p.bs[li] * a0;
      out[s] = out[s] / (lam0 * lam0);
    }
  }
}

// Reduction over the cluster of a half-step's values v (see the file
// comment).  cand: bit s set if owned index s may be chosen.  kd dot
// products with the columns of Xd (kd = 0: none); the candidate pivot data
// come from row idx of F (r values) and of X (kx values) and the symbol.
// Results: sh.idx (-1 if no candidate), sh.val, sh.sumsq, sh.dots[0..kd),
// sh.vec, sh.craw[0..kx), sh.piv_a, sh.piv_b.
template <typename T, int RPT>
__device__ __forceinline__ void bx_reduce(const BxProb<T>& p, const T (&v)[RPT], unsigned cand,
                                          const BxSrc<T>& Xd, int kd, const BxSrc<T>& F, const BxSrc<T>& X,
                                          int kx, int cs, int& par, BxShared<T>& sh) {
  using Mg = BxMsg<T>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = p.row0 + tid;
  T babs = T(-1), bval = T(0), ssq = T(0);
  int bidx = INT_MAX;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    ssq += v[s] * v[s];
    if ((cand >> s) & 1u) {
      const T av = fabs(v[s]);
      const int j = base + s * BX_NT;
      if (bx_better(av, j, babs, bidx)) { babs = av; bidx = j; bval = v[s]; }
    }
  }
  bx_warp_argmax(babs, bidx, bval);
  ssq = bx_warp_sum(ssq);
  // the warp's candidate pivot data: loads issued now, stored after the dot
  // products below, so that their latency overlaps the reductions
  constexpr int CV = (BX_CAND + 31) / 32;
  const int ncand = p.r + kx + 2;
  T cv[CV];
#pragma unroll
  for (int u = 0; u < CV; ++u) {
    const int w = lane + 32 * u;
    cv[u] = T(0);
    if (bidx != INT_MAX && w < ncand) {
      const int li = bidx - p.row0;  // the warp's candidate is one of the CTA's indices
      if (w < p.r) cv[u] = bx_at(p, F, w, li);
      else if (w < p.r + kx) cv[u] = bx_at(p, X, w - p.r, li);
      else cv[u] = (w == p.r + kx) ? p.as[li] : p.bs[li];
    }
  }
  // dot products with the columns of Xd, 16 at a time
  for (int l0 = 0; l0 < kd; l0 += 16) {
    T acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = T(0);
    if (l0 + 16 <= Xd.ns || l0 >= Xd.ns) {  // the chunk is all shared or all global
      const bool shd = l0 < Xd.ns;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int l = l0 + i;
        if (l < kd) {
          const T* Xc = shd ? Xd.s + (size_t)l * p.SP + tid : Xd.g + (size_t)l * p.ld + base;
#pragma unroll
          for (int s = 0; s < RPT; ++s)
            if (base + s * BX_NT < p.row1) acc[i] += (shd ? Xc[s * BX_NT] : __ldcg(&Xc[s * BX_NT])) * v[s];
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int l = l0 + i;
        if (l < kd) {
#pragma unroll
          for (int s = 0; s < RPT; ++s) {
            const int li = tid + s * BX_NT;
            if (base + s * BX_NT < p.row1) acc[i] += bx_at(p, Xd, l, li) * v[s];
          }
        }
      }
    }
    const T x = bx_transpose_sum16(acc, lane);
    if (lane < 16 && l0 + lane < kd) sh.wdots[l0 + lane][warp] = x;
  }
#pragma unroll
  for (int u = 0; u < CV; ++u)
    if (bidx != INT_MAX && lane + 32 * u < ncand) sh.wcand[warp][lane + 32 * u] = cv[u];
  if (lane == 0) { sh.wabs[warp] = babs; sh.widx[warp] = bidx; sh.wval[warp] = bval; sh.wsum[warp] = ssq; }
  __syncthreads();
  // CTA reduction (warps in order) into the CTA's partial.
  constexpr int WD = Mg::WORDS;
  T* msg = p.inbox + ((size_t)par * cs + (cs > 1 ? (int)cg::this_cluster().block_rank() : 0)) * WD;
  if (warp == 0) {
    T a = lane < BX_NW ? sh.wabs[lane] : T(-1);
    int i = lane < BX_NW ? sh.widx[lane] : INT_MAX;
    T vv = lane < BX_NW ? sh.wval[lane] : T(0);
    T ss = lane < BX_NW ? sh.wsum[lane] : T(0);
    int src = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T oa = __shfl_xor_sync(0xffffffffu, a, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      const T ov = __shfl_xor_sync(0xffffffffu, vv, o);
      const int os = __shfl_xor_sync(0xffffffffu, src, o);
      if (bx_better(oa, oi, a, i)) { a = oa; i = oi; vv = ov; src = os; }
    }
    ss = bx_warp_sum(ss);
    if (lane == 0) {
      msg[Mg::ABS] = a;
      msg[Mg::VAL] = vv;
      msg[Mg::SSQ] = ss;
      msg[Mg::IDX] = (T)(i == INT_MAX ? -1 : i);
      sh.win = (i == INT_MAX) ? -1 : src;
    }
  }
  for (int l = tid; l < kd; l += BX_NT) {
    T x = T(0);
#pragma unroll
    for (int w = 0; w < BX_NW; ++w) x += sh.wdots[l][w];
    msg[Mg::DOTS + l] = x;
  }
  __syncthreads();
  {
    const int wsrc = sh.win;
    if (wsrc >= 0)
      for (int w = tid; w < p.r + kx + 2; w += BX_NT) msg[Mg::CAND + w] = sh.wcand[wsrc][w];
  }
  if (cs > 1) {
    // push the partial into every CTA's inbox (slot = this rank), then reduce
    // the cs partials in rank order
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    const int live = Mg::CAND + p.r + kx + 2;
    __syncthreads();
    for (int i = tid; i < cs * live; i += BX_NT) {
      const int dst = i / live, w = i - dst * live;
      if (dst != me && (w < Mg::DOTS + kd || w >= Mg::CAND)) *cl.map_shared_rank(&msg[w], dst) = msg[w];
    }
    cl.sync();
    if (tid == 0) {
      T a = T(-1), vv = T(0), ss = T(0);
      int i = INT_MAX, src = -1;
      for (int qq = 0; qq < cs; ++qq) {
        const T* mq = p.inbox + ((size_t)par * cs + qq) * WD;
        ss += mq[Mg::SSQ];
        const int iq = (int)mq[Mg::IDX];
        if (iq >= 0 && bx_better(mq[Mg::ABS], iq, a, i)) { a = mq[Mg::ABS]; i = iq; vv = mq[Mg::VAL]; src = qq; }
      }
      sh.idx = src < 0 ? -1 : i;
      sh.val = vv;
      sh.sumsq = ss;
      sh.win = src;
    }
    for (int l = tid; l < kd; l += BX_NT) {
      T x = T(0);
      for (int qq = 0; qq < cs; ++qq) x += p.inbox[((size_t)par * cs + qq) * WD + Mg::DOTS + l];
      sh.dots[l] = x;
    }
    __syncthreads();
    const int src = sh.win;
    if (src >= 0) {
      const T* mq = p.inbox + ((size_t)par * cs + src) * WD;
      for (int w = tid; w < p.r + kx + 2; w += BX_NT) {
        const T x = mq[Mg::CAND + w];
        if (w < p.r) sh.vec[w] = x;
        else if (w < p.r + kx) sh.craw[w - p.r] = x;
        else if (w == p.r + kx) sh.piv_a = x;
        else sh.piv_b = x;
      }
    }
  } else {
    __syncthreads();
    if (tid == 0) {
      const int i = (int)msg[Mg::IDX];
      sh.idx = i;
      sh.val = msg[Mg::VAL];
      sh.sumsq = msg[Mg::SSQ];
    }
    for (int l = tid; l < kd; l += BX_NT) sh.dots[l] = msg[Mg::DOTS + l];
    if (sh.win >= 0)
      for (int w = tid; w < p.r + kx + 2; w += BX_NT) {
        const T x = msg[Mg::CAND + w];
        if (w < p.r) sh.vec[w] = x;
        else if (w < p.r + kx) sh.craw[w - p.r] = x;
        else if (w == p.r + kx) sh.piv_a = x;
        else sh.piv_b = x;
      }
  }
  __syncthreads();
  par ^= 1;
}

template <typename T, int RPT>
__global__ void __launch_bounds__(BX_NT, 1) bcross_kernel(const BatchProb* __restrict__ P,
                                                          const int* __restrict__ list, BatchCrossParams cp) {
  __shared__ BxShared<T> sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int cs = 1, q = 0;
  if (gridDim.x > 1 && cg::this_cluster().num_blocks() > 1) {
    cs = (int)cg::this_cluster().num_blocks();
    q = (int)cg::this_cluster().block_rank();
  }
  const BatchProb& B = P[list[blockIdx.x / cs]];
  BxProb<T> p;
  p.m = B.m;
  p.r = B.r;
  p.ld = B.ldw;
  p.kcap = B.kcap;
  {
    const int S = (p.m + cs - 1) / cs;
    p.row0 = min(p.m, q * S);
    p.row1 = min(p.m, p.row0 + S);
  }
  p.Uh = static_cast<const T*>(B.Uh);
  p.Vh = static_cast<const T*>(B.Vh);
  p.C = static_cast<T*>(B.C);
  p.R = static_cast<T*>(B.R);
  p.a = static_cast<const T*>(B.sa);
  p.b = static_cast<const T*>(B.sb);
  SolveState* st = B.st;
  // shared-memory copies of the CTA's slices: the symbol always, Uh and Vh if
  // they fit in half of what is left, then as many skeleton columns as fit
  // (the same choice in every CTA of the cluster)
  extern __shared__ __align__(16) unsigned char bx_dyn[];
  {
    const int SP = BX_NT * RPT;
    const long long w = (long long)sizeof(T);
    const long long inbox = 2LL * cs * BxMsg<T>::WORDS * w;
    const long long budget = cp.smem_bytes;
    const long long fixed = inbox + 2LL * SP * w;
    const long long uvb = 2LL * SP * p.r * w;
    p.uv = cp.cache && uvb <= (budget - fixed) / 2;
    const long long left = budget - fixed - (p.uv ? uvb : 0);
    long long KS = cp.cache ? left / (2LL * SP * w) : 0;
    if (KS > p.kcap) KS = p.kcap;
    if (KS < 0) KS = 0;
    p.SP = SP;
    p.KS = (int)KS;
    T* q0 = reinterpret_cast<T*>(bx_dyn);
    p.inbox = q0; q0 += 2 * cs * BxMsg<T>::WORDS;
    T* as = q0; q0 += SP;
    T* bs = q0; q0 += SP;
    T* Us = q0; q0 += p.uv ? (size_t)SP * p.r : 0;
    T* Vs = q0; q0 += p.uv ? (size_t)SP * p.r : 0;
    p.Cs = q0; q0 += (size_t)SP * KS;
    p.Rs = q0;
    p.as = as; p.bs = bs; p.Us = Us; p.Vs = Vs;
    const int S = p.row1 - p.row0;
    for (int li = tid; li < S; li += BX_NT) {
      as[li] = p.a[p.row0 + li];
      bs[li] = p.b[p.row0 + li];
    }
    if (p.uv)
      for (int al = 0; al < p.r; ++al)
        for (int li = tid; li < S; li += BX_NT) {
          Us[(size_t)al * SP + li] = p.Uh[p.row0 + li + (size_t)al * p.ld];
          Vs[(size_t)al * SP + li] = p.Vh[p.row0 + li + (size_t)al * p.ld];
        }
  }
  __syncthreads();
  const BxSrc<T> srcU{p.Uh, p.Us, p.uv ? p.r : 0}, srcV{p.Vh, p.Vs, p.uv ? p.r : 0};
  const BxSrc<T> srcC{p.C, p.Cs, p.KS}, srcR{p.R, p.Rs, p.KS};
  const T tol2 = (T)(cp.tol * cp.tol);
  const int base = p.row0 + tid;
  unsigned own = 0;  // owned indices
#pragma unroll
  for (int s = 0; s < RPT; ++s)
    if (base + s * BX_NT < p.row1) own |= 1u << s;
  unsigned used_r = 0, used_c = 0;
  if (tid == 0) { sh.norm2 = T(0); sh.small = 0; sh.pfloor = T(0); }
  if (cs > 1) cg::this_cluster().sync();  // every CTA runs before anyone pushes into its inbox
  const T a0 = p.a[0], b0 = p.b[0];
  int par = 0;
  T v[RPT];
  bx_scores<T, RPT>(p, a0, b0, v);
  bx_reduce<T, RPT>(p, v, own, srcC, 0, srcU, srcC, 0, cs, par, sh);
  int istar = sh.idx;
  int k = 0, probe_rounds = 0, zero_rows = 0, converged = 0;
  // index s of an owned index j (or -1)
  auto slot = [&](int j) -> int {
    const int o = j - base;
    return (j >= p.row0 && j < p.row1 && o >= 0 && o % BX_NT == 0) ? o / BX_NT : -1;
  };
  while (k < p.kcap && istar >= 0) {
    // ---------------- row half-step at istar (pivot data in sh.vec, sh.craw)
    for (int l = tid; l < k; l += BX_NT) sh.cd[l] = sh.craw[l] * sh.d[l];
    __syncthreads();
    bx_eval<T, RPT>(p, srcV, srcR, k, sh, v);
    {
      const int s = slot(istar);
      if (s >= 0) used_r |= 1u << s;
    }
    bx_reduce<T, RPT>(p, v, own & ~used_c, srcR, k, srcV, srcR, k, cs, par, sh);
    const int jstar = sh.idx;
    {
      const int s = jstar >= 0 ? slot(jstar) : -1;
      if (s >= 0) used_c |= 1u << s;
    }
    if (tid == 0) {
      const T dv = jstar >= 0 ? sh.val : T(0);
      // a pivot far below the working precision's rounding noise (relative
      // to the first pivot) is a zero row
      sh.flag = !(fabs(dv) > sh.pfloor);
      sh.delta = dv;
      sh.rsq = sh.sumsq;
    }
    __syncthreads();
    if (sh.flag) {
      // the row is represented exactly: move to the best-scored unused row
      ++zero_rows;
      bx_scores<T, RPT>(p, a0, b0, v);
      bx_reduce<T, RPT>(p, v, own & ~used_r, srcC, 0, srcU, srcC, k, cs, par, sh);
      if (zero_rows > cp.max_zero_rows || sh.idx < 0) { converged = 1; break; }
      istar = sh.idx;
      continue;
    }
    // ---------------- column half-step at jstar
    const T tdelta = sh.delta;
    for (int l = tid; l < k; l += BX_NT) {
      sh.gr[l] = sh.dots[l] / tdelta;
      sh.cd[l] = sh.craw[l] * sh.d[l];
    }
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if ((own >> s) & 1u) {
        const T rv = v[s] / tdelta;
        p.R[base + s * BX_NT + (size_t)k * p.ld] = rv;
        if (k < p.KS) p.Rs[(size_t)k * p.SP + tid + s * BX_NT] = rv;
      }
    __syncthreads();
    bx_eval<T, RPT>(p, srcU, srcC, k, sh, v);
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      v[s] = v[s] / tdelta;
      if ((own >> s) & 1u) {
        p.C[base + s * BX_NT + (size_t)k * p.ld] = v[s];
        if (k < p.KS) p.Cs[(size_t)k * p.SP + tid + s * BX_NT] = v[s];
      }
    }
    if (tid == 0) sh.d[k] = tdelta;
    // the next row step needs column k of C: the winner's own value
    bx_reduce<T, RPT>(p, v, own & ~used_r, srcC, k, srcU, srcC, k, cs, par, sh);
    const int inext = sh.idx;
    // ---------------- bookkeeping (thread 0 of every CTA, same arithmetic)
    if (tid == 0) {
      if (inext >= 0) sh.craw[k] = sh.val;
      const T delta = sh.delta;
      const T csq = sh.sumsq;
      const T rr = (sh.rsq / delta) / delta;
      T csum = T(0);
      for (int l = 0; l < k; ++l) csum += sh.d[l] * sh.dots[l] * sh.gr[l];
      const T term2 = csq * sh.rsq;  // |d|^2 |c|^2 |r|^2
      sh.norm2 += T(2) * delta * csum + term2;
      sh.small = (term2 <= tol2 * sh.norm2) ? sh.small + 1 : 0;
      if (k == 0) sh.pfloor = fabs(delta) * (T)(sizeof(T) == 4 ? 1e-9 : 1e-20);
      if (q == 0) {
        B.GC[k + (size_t)k * p.kcap] = (double)csq;
        B.GR[k + (size_t)k * p.kcap] = (double)rr;
        B.d[k] = (double)delta;
        B.I[k] = istar;
        B.J[k] = jstar;
      }
    }
    if (q == 0)
      for (int l = tid; l < k; l += BX_NT) {
        const double gc = (double)sh.dots[l], gr = (double)sh.gr[l];
        B.GC[l + (size_t)k * p.kcap] = gc;
        B.GC[k + (size_t)l * p.kcap] = gc;
        B.GR[l + (size_t)k * p.kcap] = gr;
        B.GR[k + (size_t)l * p.kcap] = gr;
      }
    __syncthreads();
    ++k;
    if (sh.small >= 2) {
      if (probe_rounds >= cp.max_probe_rounds || cp.probes <= 0) { converged = 1; break; }
      // residual probes at splitmix64-drawn entries; probe pr on warp pr mod
      // (warps per CTA), the same arithmetic in every CTA
      const int Pn = cp.probes < 32 ? cp.probes : 32;
      for (int pr = warp; pr < Pn; pr += BX_NW) {
        const unsigned long long z = bx_splitmix64_at(cp.seed + (unsigned long long)probe_rounds,
                                                      (unsigned long long)(pr + 1));
        const int pi = (int)((z >> 32) % (unsigned long long)p.m);
        const int pj = (int)((z & 0xFFFFFFFFULL) % (unsigned long long)p.m);
        double num = 0.0, sk = 0.0;
        for (int al = lane; al < p.r; al += 32)
          num += (double)p.Uh[pi + (size_t)al * p.ld] * (double)p.Vh[pj + (size_t)al * p.ld];
        for (int l = lane; l < k; l += 32)
          sk += (double)__ldcg(&p.C[pi + (size_t)l * p.ld]) * (double)sh.d[l] *
                (double)__ldcg(&p.R[pj + (size_t)l * p.ld]);
        num = bx_warp_sum(num);
        sk = bx_warp_sum(sk);
        const double den = (double)p.a[pi] * (double)p.b[pj] + (double)p.b[pi] * (double)p.a[pj];
        if (lane == 0) { sh.probe[pr] = fabs(num / den - sk); sh.probe_row[pr] = pi; }
      }
      __syncthreads();
      if (tid == 0) {
        double worst = -1.0;
        int wrow = -1;
        for (int pr = 0; pr < Pn; ++pr)
          if (sh.probe[pr] > worst) { worst = sh.probe[pr]; wrow = sh.probe_row[pr]; }
        const double n2 = (double)sh.norm2;
        sh.flag = worst <= cp.tol * sqrt(n2 > 0.0 ? n2 : 0.0) ? -1 : wrow;
        if (sh.flag >= 0) sh.small = 0;
      }
      __syncthreads();
      ++probe_rounds;
      const int bad_row = sh.flag;
      if (bad_row < 0) { converged = 1; break; }
      // restart at the bad probe's row if unused, else at the best unused score
      bx_scores<T, RPT>(p, a0, b0, v);
      {
        const int s = slot(bad_row);
        if (s >= 0 && !((used_r >> s) & 1u)) {
#pragma unroll
          for (int ss = 0; ss < RPT; ++ss)
            if (ss == s) v[ss] = T(INFINITY);
        }
      }
      bx_reduce<T, RPT>(p, v, own & ~used_r, srcC, 0, srcU, srcC, k, cs, par, sh);
      istar = sh.idx;
      if (istar < 0) { converged = 1; break; }
      continue;
    }
    istar = inext;
    if (istar < 0) { converged = 1; break; }
  }
  // no CTA may exit while another can still write into its shared memory
  if (cs > 1) cg::this_cluster().sync();
  if (q == 0 && tid == 0) {
    st->k = k;
    st->converged = converged;
    st->probe_rounds = probe_rounds;
    st->zero_rows = zero_rows;
    st->norm2 = (double)sh.norm2;
  }
}

template <typename T, int RPT>
cudaError_t launch_bcross_rpt(const BatchProb* probs, const int* list, int n, int cs,
                              const BatchCrossParams& cp, cudaStream_t st) {
  auto kern = bcross_kernel<T, RPT>;
  // dynamic shared memory: what the SM has left beside the static part
  static int dyn = 0;
  static cudaError_t attr = [&] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess) {
      dyn = optin - (int)fa.sharedSizeBytes - 1024;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  BatchCrossParams c2 = cp;
  c2.smem_bytes = dyn;
  // without the factor cache only the inbox and the symbol slices are needed
  const size_t need = c2.cache ? (size_t)dyn
                               : ((size_t)2 * cs * BxMsg<T>::WORDS + 2 * (size_t)BX_NT * RPT) * sizeof(T);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * cs), 1, 1);
  cfg.blockDim = dim3(BX_NT, 1, 1);
  cfg.dynamicSmemBytes = need;
  cfg.stream = st;
  cudaLaunchAttribute attr_[1];
  attr_[0].id = cudaLaunchAttributeClusterDimension;
  attr_[0].val.clusterDim.x = cs;
  attr_[0].val.clusterDim.y = 1;
  attr_[0].val.clusterDim.z = 1;
  cfg.attrs = attr_;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, probs, list, c2);
}

}  // namespace

int batch_cross_max_rows(bool f32) { return BX_NT * (f32 ? 32 : 16); }

template <typename T>
cudaError_t launch_batch_cross(const BatchProb* probs, const int* list, int n, int cs, int rows_per_cta,
                               const BatchCrossParams& cp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (cs != 1 && cs != 2 && cs != 4 && cs != 8 && cs != 16) return cudaErrorInvalidValue;
  const int rpt = (rows_per_cta + BX_NT - 1) / BX_NT;
  if (rpt <= 4) return launch_bcross_rpt<T, 4>(probs, list, n, cs, cp, st);
  if (rpt <= 8) return launch_bcross_rpt<T, 8>(probs, list, n, cs, cp, st);
  if (rpt <= 16) return launch_bcross_rpt<T, 16>(probs, list, n, cs, cp, st);
  if constexpr (sizeof(T) == 4) {
    if (rpt <= 32) return launch_bcross_rpt<T, 32>(probs, list, n, cs, cp, st);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_batch_cross<float>(const BatchProb*, const int*, int, int, int, const BatchCrossParams&,
                                               cudaStream_t);
template cudaError_t launch_batch_cross<double>(const BatchProb*, const int*, int, int, int,
                                                const BatchCrossParams&, cudaStream_t);

}  // namespace lrp
