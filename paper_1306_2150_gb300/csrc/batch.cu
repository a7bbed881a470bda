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
// FFT, chirp):
//   M <= 4096 : one item = 4096 / M columns of one problem, whole sequences in
//               shared memory (Stockham passes, tiles of 4096 elements);
//   M >  4096 : float32 batches with enough columns: the one-pass transform,
//               one CTA per column, the length-M convolution split into
//               residue classes of FFTs held whole in shared memory (in-place
//               stages, fft_inplace.cuh), no scratch; otherwise the four-step
//               split M = M1 M2 through the problem's global scratch (column
//               pass, row pass with the spectrum product, column pass).
//
// Cross (Section 4.2, Eq. flr:div): one CTA, or a cluster of 2 to 16 CTAs, per
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
#include <type_traits>

#include "fft_common.cuh"
#include "fft_inplace.cuh"
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

// The fields of a problem that column addressing reads, loaded once (a
// kernel that addresses many columns of one problem keeps them in registers
// instead of reading the problem record again for every column).
struct ColGeom {
  int r, ncap, rank, ld_in, ldw, ld_out;
  const double* U;
  const double* V;
  double* Uo;
  double* Vo;
  void* Uh;
  void* Vh;
  const void* W;
  ColGeom() = default;
  __device__ __forceinline__ ColGeom(const BatchProb& B, bool with_rank) {
    r = B.r; ncap = B.ncap; ld_in = B.ld_in; ldw = B.ldw; ld_out = B.ld_out;
    U = B.U; V = B.V; Uo = B.Uo; Vo = B.Vo; Uh = B.Uh; Vh = B.Vh; W = B.W;
    rank = with_rank ? B.st->rank : 0;
  }
};

// Column addressing of a batched transform.  dir 0: column c < 2r of
// [U V] -> [Uh Vh]; dir 1: column c < 2 ncap of W -> [Uo Vo], live while its
// index within its factor is below the kept rank.
template <typename T, int DIR>
struct BCol {
  const void* in = nullptr;
  void* out = nullptr;
  bool live = false;
  BCol() = default;
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
  __device__ __forceinline__ BCol(const ColGeom& G, int col) {
    if (DIR == 0) {
      const int seg = col < G.r ? 0 : 1, cc = col - seg * G.r;
      live = col < 2 * G.r;
      in = (seg ? G.V : G.U) + (size_t)cc * G.ld_in;
      out = static_cast<T*>(seg ? G.Vh : G.Uh) + (size_t)cc * G.ldw;
    } else {
      const int seg = col < G.ncap ? 0 : 1, cc = col - seg * G.ncap;
      live = col < 2 * G.ncap && cc < G.rank;
      in = static_cast<const T*>(G.W) + (size_t)col * G.ldw;
      out = (seg ? G.Vo : G.Uo) + (size_t)cc * G.ld_out;
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
  // out[t] as stored (read back by the thread that stored it)
  __device__ __forceinline__ T loadout(int t) const {
    if (DIR == 0) return static_cast<const T*>(out)[t];
    return (T)static_cast<const double*>(out)[t];
  }
};

// Column of the inverse transform for dense live index c (0 <= c < 2R:
// U columns 0..R-1, then V columns ncap..ncap+R-1), -1 past the live ones.
__device__ __forceinline__ int live_col(const BatchProb& B, int c) {
  const int R = B.st->rank;
  return c < R ? c : (c < 2 * R ? B.ncap + (c - R) : -1);
}

__device__ __forceinline__ int live_col(const ColGeom& G, int c) {
  const int R = G.rank;
  return c < R ? c : (c < 2 * R ? G.ncap + (c - R) : -1);
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

// The contiguous range of items of this CTA (items of one problem are
// contiguous, so a CTA looks its problem up once and then steps through the
// prefix table instead of searching it for every item).
struct ItemRange {
  int begin, end, q, qbeg, qend;  // qbeg, qend: the items of problem q
  __device__ __forceinline__ ItemRange(const BatchItems& it, int items) {
    const int per = (items + (int)gridDim.x - 1) / (int)gridDim.x;
    begin = min(items, (int)blockIdx.x * per);
    end = min(items, begin + per);
    q = -1;
    qbeg = qend = 0;
  }
  __device__ __forceinline__ int problem(const BatchItems& it, int item) {
    if (q < 0) {
      q = it.live ? find_live_item(it, item) : find_item(it.start, it.n, item);
      qbeg = __ldcg(&it.start[q]);
      qend = __ldcg(&it.start[q + 1]);
    }
    while (item >= qend) {  // uniform across the CTA
      ++q;
      qbeg = qend;
      qend = __ldcg(&it.start[q + 1]);
    }
    return q;
  }
};

constexpr int kBTile = 4096;          // complex elements per tile
constexpr int kBThreads = kBTile / EPT;


// ---- M <= 4096: whole sequences in shared memory ---------------------------
template <typename T, int DIR>
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) bdst_small_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                               const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);  // padded tile (smem_ix<true>)
  cpx<T>* stw = buf + kBTile + (kBTile >> 4);
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  const int items = item_count(it);
  ItemRange rg(it, items);
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    const BatchProb& B = P[it.list[q]];
    const int logM = B.logM, M = 1 << logM, lognf = 12 - logM;
    const int col0 = (item - rg.qbeg) << lognf;
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
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) bdst_col_fwd_kernel(const BatchProb* __restrict__ P, BatchItems it,
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
  ItemRange rg(it, items);
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2;
    const int logTX = 12 - logM2, TX = 1 << logTX;
    const int bpc = (1 << logM1) >> logTX;
    const int local = item - rg.qbeg;
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
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) bdst_row_mid_kernel(const BatchProb* __restrict__ P, BatchItems it,
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
  ItemRange rg(it, items);
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2, M1 = 1 << logM1;
    const int logRY = 12 - logM1;
    const int bpc = (1 << logM2) >> logRY;
    const int local = item - rg.qbeg;
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
__global__ void __launch_bounds__(kBThreads, sizeof(T) == 4 ? 2 : 1) bdst_col_inv_kernel(const BatchProb* __restrict__ P, BatchItems it,
                                                                 const cpx<T>* __restrict__ tw4096) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* stw = buf + kBTile + 512;  // after the (row pass: padded) tile
  build_stage_twiddles(stw, tw4096, 12, it.slog);
  const int stride = stage_stride(it.slog);
  const int items = item_count(it);
  ItemRange rg(it, items);
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    const BatchProb& B = P[it.list[q]];
    const int logM1 = B.logM1, logM2 = B.logM2;
    const int logTX = 12 - logM2, TX = 1 << logTX;
    const int bpc = (1 << logM1) >> logTX;
    const int local = item - rg.qbeg;
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

// ---- M > 4096, one pass per column: Bluestein's convolution of length M
// split into R = M / H residue classes of the frequency index, H = min(M,
// 2^LH), each a length-H FFT held whole in shared memory (fft_inplace.cuh).
// With a_j = x_j chirp_j (j < m <= M / 2) and w_M = exp(-2 pi i / M):
//   A[R k + t] = FFT_H( sum_q a_(j + qH) w_M^((j + qH) t) )[k]       (fold)
//   z_j = sum_t w_M^(-j t) IFFT_H( A[R k + t] bhat[R k + t] )[j mod H]
// (IFFT unnormalised), out_j = Im(chirp_j z_j) accumulated over t in the
// output column itself.  The fold is the first forward stage's load, the
// spectrum product sits between the last forward and the first inverse
// stage in registers, and the last inverse stage writes the output: the
// column is read R times (from L2) and no M-length scratch passes through
// memory.  R = 1 for M <= 2^LH, where an item holds 2^LH / M columns.
template <typename T> __host__ __device__ constexpr int fused_logh() { return kFusedLogH32; }
// 512 threads: two radix-16 butterflies per thread and stage in float32, one
// in float64 (up to 128 registers per thread)
template <typename T> __host__ __device__ constexpr int fused_threads() { return (1 << fused_logh<T>()) / 16; }
// CTAs per SM: two when a CTA's shared memory allows (one CTA's global-memory
// waits between its barrier-separated stages then overlap the other's work)
template <typename T> __host__ __device__ constexpr int fused_ctas_per_sm() {
  return fused_logh<T>() <= 13 ? 2 : 1;
}

template <typename T>
__host__ __device__ constexpr size_t fused_smem_elems() {
  return (size_t)(1 << fused_logh<T>()) + (1 << (fused_logh<T>() - 4)) + inplace_tab_elems(fused_logh<T>()) +
         kTwHi + kTwLo;
}

// The stages of one residue t of one item, sequences of length 2^LOGH.
template <typename T, int DIR, int LOGH>
__device__ __forceinline__ void fused_residue(cpx<T>* buf, const cpx<T>* tab, const cpx<T>* th, const cpx<T>* tl,
                                              const ColGeom& G, const BatchItems& it, int col0, int m, int logM,
                                              int t, const cpx<T>* __restrict__ chirp,
                                              const cpx<T>* __restrict__ spec, int pf_col0) {
  constexpr int LH = fused_logh<T>(), HX = 1 << LH, NT = fused_threads<T>();
  constexpr int H = 1 << LOGH, LOGS0 = LOGH - 4, S0 = 1 << LOGS0;
  constexpr int N16 = LOGH >> 2, REM = LOGH & 3;
  constexpr int NMID = REM ? N16 : N16 - 1;  // radix-16 stages before the last stage
  const int M = 1 << logM;
  __syncthreads();  // tables and G written; the previous residue read buf
  // first forward stage, its elements folded from the input columns
#pragma unroll
  for (int g0 = 0; g0 < (HX >> 4); g0 += NT) {
    const int g = g0 + (int)threadIdx.x;
    const int f = g >> LOGS0, j = g & (S0 - 1);
    const int lc = col0 + f;
    const int cl = it.live ? live_col(G, lc) : lc;
    const BCol<T, DIR> c(G, cl < 0 ? 2 * G.ncap : cl);
    if (DIR == 0 && pf_col0 >= 0) {
      // the CTA's next column (same problem) into L2 while this one runs:
      // the forward input is read from HBM, the inverse one is already in L2
      const BCol<T, DIR> cn(G, pf_col0 + f);
      if (cn.live)
        for (int e0 = 0; e0 < m; e0 += H)
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int e = e0 + j + u * S0;
            if (e < m) asm volatile("prefetch.global.L2 [%0];" ::"l"(static_cast<const double*>(cn.in) + e));
          }
    }
    cpx<T> x[16], a[3], b[3];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = {T(0), T(0)};
    if (c.live)
      for (int e0 = 0; e0 < m; e0 += H) {  // uniform; once unless m > H
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int e = e0 + j + u * S0;
          if (e < m) {
            const T xv = c.load(e);
            const cpx<T> w = chirp[e];
            cpx<T> av = {xv * w.re, xv * w.im};
            if (t > 0) av = cmul(av, twiddle2(th, tl, (t * e) & (M - 1)));
            x[u] = cadd(x[u], av);
          }
        }
      }
    stage_twiddles(tab, S0, j, a, b);
    dif16(x, a, b);
    cpx<T>* bp = buf + smem_ix<true>((f << LOGH) + j);
#pragma unroll
    for (int u = 0; u < 16; ++u) bp[pad_off(u * S0)] = x[u];
  }
  if constexpr (NMID > 1) {
    __syncthreads();
    inplace_stage16c<T, false, NT, LH, LOGH - 8>(buf, tab + inplace_tab_offset(LOGH, 1));
  }
  if constexpr (NMID > 2) {
    __syncthreads();
    inplace_stage16c<T, false, NT, LH, LOGH - 12>(buf, tab + inplace_tab_offset(LOGH, 2));
  }
  static_assert(NMID <= 3, "at most four radix-16 stages");
  __syncthreads();
  inplace_last<T, REM == 2 ? 4 : (REM == 1 ? 2 : 16), NT, HX>(buf, LOGH, spec);
  if constexpr (NMID > 2) {
    __syncthreads();
    inplace_stage16c<T, true, NT, LH, LOGH - 12>(buf, tab + inplace_tab_offset(LOGH, 2));
  }
  if constexpr (NMID > 1) {
    __syncthreads();
    inplace_stage16c<T, true, NT, LH, LOGH - 8>(buf, tab + inplace_tab_offset(LOGH, 1));
  }
  __syncthreads();
  // last inverse stage, its elements written to the output columns
#pragma unroll
  for (int g0 = 0; g0 < (HX >> 4); g0 += NT) {
    const int g = g0 + (int)threadIdx.x;
    const int f = g >> LOGS0, j = g & (S0 - 1);
    const int lc = col0 + f;
    const int cl = it.live ? live_col(G, lc) : lc;
    const BCol<T, DIR> c(G, cl < 0 ? 2 * G.ncap : cl);
    const cpx<T>* bp = buf + smem_ix<true>((f << LOGH) + j);
    cpx<T> x[16], a[3], b[3];
    // the earlier residues' sums: loaded before the butterfly (float32;
    // float64 has no registers to spare for them there)
    constexpr bool early = sizeof(T) == 4;
    T old[16];
    if (early && t > 0) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int k = j + u * S0;
        old[u] = c.live && k < m ? c.loadout(k) : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = bp[pad_off(u * S0)];
    stage_twiddles(tab, S0, j, a, b);
    dit16(x, a, b);
    if (!c.live) continue;
    for (int e0 = 0; e0 < m; e0 += H) {  // uniform; once unless m > H
      if (t > 0 && (e0 > 0 || !early)) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int k = e0 + j + u * S0;
          old[u] = k < m ? c.loadout(k) : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int k = e0 + j + u * S0;
        if (k < m) {
          cpx<T> z = x[u];
          if (t > 0) z = cmulc(z, twiddle2(th, tl, (t * k) & (M - 1)));  // times w_M^(-k t)
          const cpx<T> w = chirp[k];
          const T val = w.re * z.im + w.im * z.re;  // Im(chirp z)
          c.store(k, t > 0 ? old[u] + val : val);
        }
      }
    }
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(fused_threads<T>(), fused_ctas_per_sm<T>()) bdst_fused_kernel(const BatchProb* __restrict__ P,
                                                                          BatchItems it) {
  constexpr int LH = fused_logh<T>(), HX = 1 << LH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);  // padded (smem_ix<true>)
  cpx<T>* tab = buf + HX + (HX >> 4);                  // radix-16 stage twiddles
  cpx<T>* th = tab + inplace_tab_elems(LH);            // w_M two-level tables
  cpx<T>* tl = th + kTwHi;
  __shared__ ColGeom sg[2];  // column geometry of the current item (by item parity)
  int curM = 0;
  const int items = item_count(it);
  ItemRange rg(it, items);
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    const BatchProb& B = P[it.list[q]];
    const int logM = B.logM;
    const int logH = logM < LH ? logM : LH;
    const int R = 1 << (logM - logH), lognf = LH - logH;
    const int col0 = (item - rg.qbeg) << lognf;
    if (threadIdx.x == 0) sg[item & 1] = ColGeom(B, DIR == 1);  // read after the next barrier
    const ColGeom& G = sg[item & 1];
    if (logM != curM) {  // uniform across the CTA
      __syncthreads();   // the previous item read the tables
      const cpx<T>* tw = static_cast<const cpx<T>*>(B.tw);
      load_twiddles2(th, tl, tw, logM);
      build_inplace_tables(tab, tw, logM, logH);
      curM = logM;
    }
    const cpx<T>* chirp = static_cast<const cpx<T>*>(B.chirp);
    const cpx<T>* bres = static_cast<const cpx<T>*>(B.bres);
    const int m = B.m;
    // next column of the same problem in this CTA's range: prefetched in the first residue
    const int pf = item + 1 < rg.end && item + 1 < rg.qend ? col0 + (1 << lognf) : -1;
    for (int t = 0; t < R; ++t) {  // uniform
      const cpx<T>* spec = bres + ((size_t)t << logH);
      const int pft = t == 0 ? pf : -1;
      if (logH == LH) fused_residue<T, DIR, LH>(buf, tab, th, tl, G, it, col0, m, logM, t, chirp, spec, pft);
      else fused_residue<T, DIR, LH - 1>(buf, tab, th, tl, G, it, col0, m, logM, t, chirp, spec, pft);
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
  if (col.items > 0 && col.fused_logh) {
    if constexpr (sizeof(T) != 4) {
      return cudaErrorInvalidValue;  // float32 only
    } else {
      if (col.fused_logh != fused_logh<T>()) return cudaErrorInvalidValue;
      auto kf = bdst_fused_kernel<T, DIR>;
      const size_t fbytes = fused_smem_elems<T>() * sizeof(cpx<T>);
      static cudaError_t fattr =
          cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fbytes);
      if (fattr != cudaSuccess) return fattr;
      // one or two CTAs per SM (the whole sequence in shared memory)
      const int cap = fused_ctas_per_sm<T>() * num_sms;
      kf<<<col.items < cap ? col.items : cap, fused_threads<T>(), fbytes, st>>>(probs, col);
      return cudaGetLastError();
    }
  }
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
      } else if (kind == 1 && it.fused_logh) {
        const int nf = 1 << (it.fused_logh - min(B.logM, it.fused_logh));
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
// thread per row, both factors; Tc and Tr staged in shared memory once per
// problem of the CTA's item range.
// ---------------------------------------------------------------------------
namespace {
template <typename T>
__global__ void __launch_bounds__(256) brotate_kernel(const BatchProb* __restrict__ P, BatchItems it) {
  extern __shared__ __align__(16) unsigned char rot_raw[];
  // rotations transposed, [side][l][q] (q contiguous, zero past the rank), so
  // that the 16 coefficients of a row l are four (float32) or eight (float64)
  // vector loads that every thread of the CTA shares
  T* tm = reinterpret_cast<T*>(rot_raw);
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int VW = (int)(sizeof(V) / sizeof(T));
  const int items = item_count(it);
  ItemRange rg(it, items);
  int lastq = -1, k = 0, R = 0, m = 0, ldw = 0;
  const T* Xs[2] = {nullptr, nullptr};
  T* W = nullptr;
  size_t side_off = 0;
  for (int item = rg.begin; item < rg.end; ++item) {
    const int q = rg.problem(it, item);
    if (q != lastq) {  // a new problem: its sizes, and its rotations staged
      const BatchProb& B = P[it.list[q]];
      k = B.st->k;
      R = B.st->rank;
      m = B.m;
      ldw = B.ldw;
      Xs[0] = static_cast<const T*>(B.C);
      Xs[1] = static_cast<const T*>(B.R);
      W = static_cast<T*>(B.W);
      side_off = (size_t)B.ncap * B.ldw;
      __syncthreads();  // the previous problem's rows read tm
      const int R16 = (R + 15) & ~15;
      if (R > 0 && k > 0)
        for (int idx = threadIdx.x; idx < k * R16; idx += blockDim.x) {
          const int qq = idx % R16, l = idx / R16;
          const bool in = qq < R;
          tm[l * KMAX + qq] = in ? static_cast<const T*>(B.Tc)[l + (size_t)qq * KMAX] : T(0);
          tm[KMAX * KMAX + l * KMAX + qq] = in ? static_cast<const T*>(B.Tr)[l + (size_t)qq * KMAX] : T(0);
        }
      __syncthreads();
      lastq = q;
    }
    if (R <= 0 || k <= 0) continue;
    const int row = ((item - rg.qbeg) << 8) + threadIdx.x;
    if (row >= m) continue;
    for (int side = 0; side < 2; ++side) {
      const T* X = Xs[side] + row;
      const T* ts = tm + side * KMAX * KMAX;
      T* out = W + side * side_off + row;
      for (int q0 = 0; q0 < R; q0 += 16) {  // one pass over X for ranks up to 16
        T acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = T(0);
#pragma unroll 4
        for (int l = 0; l < k; ++l) {
          const T x = X[(size_t)l * ldw];
          const V* tv = reinterpret_cast<const V*>(ts + l * KMAX + q0);
#pragma unroll
          for (int v = 0; v < 16 / VW; ++v) {
            const V c4 = tv[v];
            if constexpr (VW == 4) {
              acc[4 * v] += x * c4.x;
              acc[4 * v + 1] += x * c4.y;
              acc[4 * v + 2] += x * c4.z;
              acc[4 * v + 3] += x * c4.w;
            } else {
              acc[2 * v] += x * c4.x;
              acc[2 * v + 1] += x * c4.y;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (q0 + c < R) out[(size_t)(q0 + c) * ldw] = acc[c];
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
// Batched cross.  Every thread of the cluster holds the state of the cross
// (step, pivots, norm estimate, stop counters) in registers and takes every
// decision itself from reductions whose results are identical in every warp
// and every CTA, so no decision is broadcast:
//   1. residual entries of the owned indices (F = Uh or Vh, X = C or R);
//   2. warp partials -- argmax (lowest index on ties), sum of squares, dot
//      products with the columns of X, and the pivot data of the warp's own
//      candidate (its rows of F and X and its symbol) -- into a slot per warp;
//   3. CTA barrier; warp 0 combines the slots in warp order;
//   4. cluster: warp 0 pushes the CTA result into a slot per CTA in every
//      CTA's inbox (distributed shared memory); cluster barrier; warp 0
//      combines the inbox in rank order;
//   5. warp 0 writes the combined result to shared memory; CTA barrier;
//      every warp reads it.
// Slots, inboxes and results alternate between two buffers, so a buffer is
// rewritten only after a barrier that every reader of its previous contents
// has passed.
// ---------------------------------------------------------------------------
namespace {

constexpr int BX_NT = 512;            // threads per CTA
constexpr int BX_NW = BX_NT / 32;
constexpr int BX_CAND = 2 * KMAX + 3; // pivot data: a, b, F row (<= KMAX), X row (<= KMAX)
// words of a slot: header, dot products, pivot data
constexpr int BX_ABS = 0, BX_VAL = 1, BX_SSQ = 2, BX_IDX = 3, BX_DOTS = 4, BX_CND = BX_DOTS + KMAX;
constexpr int BX_WORDS = BX_CND + BX_CAND;
constexpr int BX_RES = 4 + KMAX;  // result words: index, value, sum of squares, winner slot, dots

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

// argmax over the warp carrying the value and a source tag
template <typename T>
__device__ __forceinline__ void bx_warp_argmax(T& a, int& i, T& v, int& src) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T oa = __shfl_xor_sync(0xffffffffu, a, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int os = __shfl_xor_sync(0xffffffffu, src, o);
    if (bx_better(oa, oi, a, i)) { a = oa; i = oi; v = ov; src = os; }
  }
}

template <typename T> __device__ __forceinline__ T bx_ratio(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float bx_ratio<float>(float a, float b) { return __fdividef(a, b); }

// Two CTAs per SM (64 registers per thread) for float32 slices of up to 8
// indices per thread, so that a batch of many problems on a few CTAs each
// runs in one wave; one CTA per SM (128 registers) otherwise.
template <typename T, int RPT>
__host__ __device__ constexpr bool bx_two_per_sm() { return sizeof(T) == 4 && RPT <= 8; }

// Sum over the warp of a[i], i < DC, for every i at once (recursive halving);
// afterwards lane L holds the sum for index L mod DC.  Fixed pattern: every
// warp and CTA gets the same bits.
template <int DC, typename T>
__device__ __forceinline__ T bx_transpose_sum(T (&a)[DC], int lane) {
#pragma unroll
  for (int h = DC / 2; h >= 1; h >>= 1) {
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
  for (int h = DC; h < 32; h <<= 1) x += __shfl_xor_sync(0xffffffffu, x, h);
  return x;  // sum of value (lane mod DC) over the warp
}

// Problem-level constants of one CTA: owned indices j = row0 + tid + s NT.
template <typename T>
struct BxProb {
  int m, r, ld, kcap, row0, row1, cs, rank;
  bool full;  // all RPT indices of this thread are in its CTA's slice
  const T* Uh;
  const T* Vh;
  T* C;
  T* R;
  const T* a;
  const T* b;
  T* slots;   // [2][NW][BX_WORDS]
  T* inbox;   // [2][cs][BX_WORDS]
  T* res;     // [2][BX_RES]: the CTA's combined result
};

// Result of a reduction, identical in every thread of the cluster.
template <typename T>
struct BxRed {
  int idx;          // winning index (-1: no candidate)
  T val, ssq;
  T dlo, dhi;       // dot products l = lane and l = lane + 32 (this lane's)
  const T* cand;    // pivot data of the winner: a, b, F row, X row
};

// Pivot data of the next half-step: cand (a, b, F row, X row of kx entries)
// and, if ext, one more X entry xv (the column the step just built).
template <typename T>
struct BxPivot {
  const T* cand;
  int kx;
  int ext;
  T xv;
};

// out[s] = (vec . F[j]) / (pa b_j + pb a_j) - sum_{l<k} craw[l] d[l] X[j, l]
// for the owned indices (0 elsewhere); vec, craw, pa, pb from the pivot data.
// Index s of the thread is in its CTA's slice (always, for FULL threads).
template <bool FULL, typename T>
__device__ __forceinline__ bool bx_in(const BxProb<T>& p, int base, int s) {
  return FULL || base + s * BX_NT < p.row1;
}

template <typename T, int RPT, bool FULL>
__device__ __forceinline__ void bx_eval_t(const BxProb<T>& p, const T* __restrict__ F, const T* __restrict__ X, int k,
                                          const BxPivot<T>& pv, const T* d, T (&out)[RPT]) {
  const int base = p.row0 + threadIdx.x;
  const T* vec = pv.cand + 2;
#pragma unroll
  for (int s = 0; s < RPT; ++s) out[s] = T(0);
#pragma unroll 8
  for (int al = 0; al < p.r; ++al) {
    const T w = vec[al];
    const T* Fc = F + (size_t)al * p.ld + base;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (bx_in<FULL>(p, base, s)) out[s] += w * __ldg(&Fc[s * BX_NT]);
  }
  const T pa = pv.cand[0], pb = pv.cand[1];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int j = base + s * BX_NT;
    out[s] = bx_in<FULL>(p, base, s) ? bx_ratio<T>(out[s], pa * __ldg(&p.b[j]) + pb * __ldg(&p.a[j])) : T(0);
  }
  const T* craw = pv.cand + 2 + p.r;
#pragma unroll 8
  for (int l = 0; l < k; ++l) {
    const T c = (l < pv.kx ? craw[l] : pv.xv) * d[l];
    const T* Xc = X + (size_t)l * p.ld + base;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (bx_in<FULL>(p, base, s)) out[s] -= c * Xc[s * BX_NT];
  }
}

// Threads whose indices all lie in the slice (every thread but the last few
// of a problem's last CTA) run the loops without per-index tests.
template <typename T, int RPT>
__device__ __forceinline__ void bx_eval(const BxProb<T>& p, const T* __restrict__ F, const T* __restrict__ X, int k,
                                        const BxPivot<T>& pv, const T* d, T (&out)[RPT]) {
  if (p.full) bx_eval_t<T, RPT, true>(p, F, X, k, pv, d, out);
  else bx_eval_t<T, RPT, false>(p, F, X, k, pv, d, out);
}

// Start score ||Uh[j]||^2 / Lambda[j, 0]^2 of the owned indices.
template <typename T, int RPT>
__device__ __forceinline__ void bx_scores(const BxProb<T>& p, T a0, T b0, T (&out)[RPT]) {
  const int base = p.row0 + threadIdx.x;
#pragma unroll
  for (int s = 0; s < RPT; ++s) out[s] = T(0);
#pragma unroll 8
  for (int al = 0; al < p.r; ++al) {
    const T* Fc = p.Uh + (size_t)al * p.ld + base;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if (base + s * BX_NT < p.row1) { const T u = __ldg(&Fc[s * BX_NT]); out[s] += u * u; }
  }
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int j = base + s * BX_NT;
    if (j < p.row1) {
      const T lam0 = __ldg(&p.a[j]) * b0 + __ldg(&p.b[j]) * a0;
      out[s] = out[s] / (lam0 * lam0);
    }
  }
}

// Reduction of a half-step's values v over the cluster (see the section
// comment).  cand: bit s set if owned index s may be chosen.  kd dot
// products with the columns of Xd; pivot data from row idx of F (r values)
// and of X (kx values).
template <typename T, int RPT>
__device__ __forceinline__ BxRed<T> bx_reduce(const BxProb<T>& p, const T (&v)[RPT], unsigned cand,
                                              const T* __restrict__ Xd, int kd, const T* __restrict__ F,
                                              const T* __restrict__ X, int kx, int& par) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = p.row0 + tid;
  T babs = T(-1), bval = T(0), ssq = T(0);
  int bidx = INT_MAX, src = 0;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    ssq += v[s] * v[s];
    if ((cand >> s) & 1u) {
      const T av = fabs(v[s]);
      const int j = base + s * BX_NT;
      if (bx_better(av, j, babs, bidx)) { babs = av; bidx = j; bval = v[s]; }
    }
  }
  bx_warp_argmax(babs, bidx, bval, src);
  ssq = bx_warp_sum(ssq);
  // the warp candidate's pivot data: loads issued now, stored after the dot
  // products so that their latency overlaps them
  constexpr int CV = (BX_CAND + 31) / 32;
  const int ncand = 2 + p.r + kx;
  T cv[CV];
#pragma unroll
  for (int u = 0; u < CV; ++u) {
    const int w = lane + 32 * u;
    cv[u] = T(0);
    if (bidx != INT_MAX && w < ncand) {
      if (w == 0) cv[u] = __ldg(&p.a[bidx]);
      else if (w == 1) cv[u] = __ldg(&p.b[bidx]);
      else if (w < 2 + p.r) cv[u] = __ldg(&F[bidx + (size_t)(w - 2) * p.ld]);
      else cv[u] = X[bidx + (size_t)(w - 2 - p.r) * p.ld];
    }
  }
  T* slot = p.slots + ((size_t)par * BX_NW + warp) * BX_WORDS;
  // dot products DC columns at a time (8 where two CTAs share an SM's
  // registers, 16 otherwise)
  constexpr int DC = bx_two_per_sm<T, RPT>() ? 8 : 16;
  auto dots = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    for (int l0 = 0; l0 < kd; l0 += DC) {
      T acc[DC];
#pragma unroll
      for (int i = 0; i < DC; ++i) {
        acc[i] = T(0);
        const int l = l0 + i;
        if (l < kd) {
          const T* Xc = Xd + (size_t)l * p.ld + base;
#pragma unroll
          for (int s = 0; s < RPT; ++s)
            if (bx_in<FULL>(p, base, s)) acc[i] += Xc[s * BX_NT] * v[s];
        }
      }
      const T x = bx_transpose_sum<DC>(acc, lane);
      if (lane < DC && l0 + lane < kd) slot[BX_DOTS + l0 + lane] = x;
    }
  };
  // the transpose sums are warp-collective: a warp with both kinds of
  // threads runs the tested loop in all of them
  if (__all_sync(0xffffffffu, p.full)) dots(std::true_type{});
  else dots(std::false_type{});
#pragma unroll
  for (int u = 0; u < CV; ++u)
    if (lane + 32 * u < ncand) slot[BX_CND + lane + 32 * u] = cv[u];
  if (lane == 0) {
    slot[BX_ABS] = babs;
    slot[BX_VAL] = bval;
    slot[BX_SSQ] = ssq;
    slot[BX_IDX] = (T)(bidx == INT_MAX ? -1 : bidx);
  }
  __syncthreads();
  // warp 0 combines the warp slots in warp order (and, in a cluster, pushes
  // the CTA result into every CTA's inbox and combines the inbox in rank
  // order) and writes the result for every warp of the CTA
  const T* sl = p.slots + (size_t)par * BX_NW * BX_WORDS;
  const T* ib = p.inbox + (size_t)par * p.cs * BX_WORDS;
  T* rs = p.res + (size_t)par * BX_RES;
  auto combine = [&](const T* base, int nq, int& i, T& a, T& vv, T& ss, int& sw, T& dlo, T& dhi) {
    a = T(-1); vv = T(0); ss = T(0); i = INT_MAX; sw = 0;
    if (lane < nq) {
      const T* q = base + (size_t)lane * BX_WORDS;
      const int qi = (int)q[BX_IDX];
      ss = q[BX_SSQ];
      if (qi >= 0) { a = q[BX_ABS]; i = qi; vv = q[BX_VAL]; }
      sw = lane;
    }
    bx_warp_argmax(a, i, vv, sw);
    ss = bx_warp_sum(ss);
    dlo = T(0);
    dhi = T(0);
    for (int w = 0; w < nq; ++w) {
      if (lane < kd) dlo += base[(size_t)w * BX_WORDS + BX_DOTS + lane];
      if (lane + 32 < kd) dhi += base[(size_t)w * BX_WORDS + BX_DOTS + lane + 32];
    }
  };
  auto publish = [&](int i, T vv, T ss, int sw, T dlo, T dhi) {
    if (lane == 0) {
      rs[0] = (T)(i == INT_MAX ? -1 : i);
      rs[1] = vv;
      rs[2] = ss;
      rs[3] = (T)sw;
    }
    if (lane < kd) rs[4 + lane] = dlo;
    if (lane + 32 < kd) rs[4 + lane + 32] = dhi;
  };
  if (warp == 0) {
    int i, sw;
    T a, vv, ss, dlo, dhi;
    combine(sl, BX_NW, i, a, vv, ss, sw, dlo, dhi);
    if (p.cs == 1) {
      publish(i, vv, ss, sw, dlo, dhi);
    } else {
      // push this CTA's result into slot `rank` of every CTA's inbox
      cg::cluster_group cl = cg::this_cluster();
      T* dst0 = p.inbox + ((size_t)par * p.cs + p.rank) * BX_WORDS;
      const T* wc = sl + (size_t)sw * BX_WORDS + BX_CND;
      for (int qd = 0; qd < p.cs; ++qd) {
        T* dq = cl.map_shared_rank(dst0, qd);
        if (lane == 0) {
          dq[BX_ABS] = a;
          dq[BX_VAL] = vv;
          dq[BX_SSQ] = ss;
          dq[BX_IDX] = (T)(i == INT_MAX ? -1 : i);
        }
        if (lane < kd) dq[BX_DOTS + lane] = dlo;
        if (lane + 32 < kd) dq[BX_DOTS + lane + 32] = dhi;
        if (i != INT_MAX)
          for (int w = lane; w < ncand; w += 32) dq[BX_CND + w] = wc[w];
      }
    }
  }
  if (p.cs > 1) {
    cg::this_cluster().sync();
    if (warp == 0) {
      int i, sw;
      T a, vv, ss, dlo, dhi;
      combine(ib, p.cs, i, a, vv, ss, sw, dlo, dhi);
      publish(i, vv, ss, sw, dlo, dhi);
    }
  }
  __syncthreads();
  BxRed<T> res;
  res.idx = (int)rs[0];
  res.val = rs[1];
  res.ssq = rs[2];
  res.dlo = lane < kd ? rs[4 + lane] : T(0);
  res.dhi = lane + 32 < kd ? rs[4 + lane + 32] : T(0);
  res.cand = (p.cs == 1 ? sl : ib) + (size_t)(int)rs[3] * BX_WORDS + BX_CND;
  par ^= 1;
  return res;
}

template <typename T, int RPT>
__global__ void __launch_bounds__(BX_NT, bx_two_per_sm<T, RPT>() ? 2 : 1) bcross_kernel(const BatchProb* __restrict__ P,
                                                          const int* __restrict__ list, BatchCrossParams cp) {
  extern __shared__ __align__(16) unsigned char bx_dyn[];
  __shared__ T sd[KMAX + 1];  // pivot values
  __shared__ double sprobe[32];
  __shared__ int sprow[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const BatchProb& B = P[list[blockIdx.x / cs]];
  BxProb<T> p;
  p.m = B.m;
  p.r = B.r;
  p.ld = B.ldw;
  p.kcap = B.kcap;
  p.cs = cs;
  p.rank = q;
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
  p.slots = reinterpret_cast<T*>(bx_dyn);
  p.inbox = p.slots + 2 * BX_NW * BX_WORDS;
  p.res = p.inbox + 2 * cs * BX_WORDS;
  SolveState* st = B.st;
  const T tol2 = (T)(cp.tol * cp.tol);
  const int base = p.row0 + tid;
  p.full = base + (RPT - 1) * BX_NT < p.row1;
  unsigned own = 0;
#pragma unroll
  for (int s = 0; s < RPT; ++s)
    if (base + s * BX_NT < p.row1) own |= 1u << s;
  unsigned used_r = 0, used_c = 0;
  auto slot = [&](int j) -> int {  // owned index slot of j, or -1
    const int o = j - base;
    return (j >= p.row0 && j < p.row1 && o >= 0 && o % BX_NT == 0) ? o / BX_NT : -1;
  };
  if (cs > 1) cl.sync();  // every CTA runs before anyone pushes into its inbox
  const T a0 = __ldg(&p.a[0]), b0 = __ldg(&p.b[0]);
  int par = 0;
  T v[RPT];
  bx_scores<T, RPT>(p, a0, b0, v);
  BxRed<T> red = bx_reduce<T, RPT>(p, v, own, p.C, 0, p.Uh, p.C, 0, par);
  int istar = red.idx;
  BxPivot<T> pv{red.cand, 0, 0, T(0)};
  int k = 0, probe_rounds = 0, zero_rows = 0, converged = 0, small = 0;
  T norm2 = T(0), pfloor = T(0);
  while (k < p.kcap && istar >= 0) {
    // ---------------- row half-step at istar
    bx_eval<T, RPT>(p, p.Vh, p.R, k, pv, sd, v);
    {
      const int s = slot(istar);
      if (s >= 0) used_r |= 1u << s;
    }
    red = bx_reduce<T, RPT>(p, v, own & ~used_c, p.R, k, p.Vh, p.R, k, par);
    const int jstar = red.idx;
    {
      const int s = jstar >= 0 ? slot(jstar) : -1;
      if (s >= 0) used_c |= 1u << s;
    }
    const T delta = jstar >= 0 ? red.val : T(0);
    // a pivot far below the working precision's rounding noise (relative to
    // the first pivot) is a zero row
    if (!(fabs(delta) > pfloor)) {
      ++zero_rows;
      bx_scores<T, RPT>(p, a0, b0, v);
      red = bx_reduce<T, RPT>(p, v, own & ~used_r, p.C, 0, p.Uh, p.C, k, par);
      if (zero_rows > cp.max_zero_rows || red.idx < 0) { converged = 1; break; }
      istar = red.idx;
      pv = {red.cand, k, 0, T(0)};
      continue;
    }
    const T rsq = red.ssq;
    const T grlo = red.dlo / delta, grhi = red.dhi / delta;  // R_l . r
    pv = {red.cand, k, 0, T(0)};
    // ---------------- column half-step at jstar
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      if ((own >> s) & 1u) p.R[base + s * BX_NT + (size_t)k * p.ld] = v[s] / delta;
    bx_eval<T, RPT>(p, p.Uh, p.C, k, pv, sd, v);
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      v[s] = v[s] / delta;
      if ((own >> s) & 1u) p.C[base + s * BX_NT + (size_t)k * p.ld] = v[s];
    }
    if (tid == 0) sd[k] = delta;  // read after the next barrier
    red = bx_reduce<T, RPT>(p, v, own & ~used_r, p.C, k, p.Uh, p.C, k, par);
    const int inext = red.idx;
    // ---------------- bookkeeping (every thread, the same arithmetic)
    {
      const T csq = red.ssq;
      const T rr = (rsq / delta) / delta;
      T part = T(0);
      if (lane < k) part += sd[lane] * red.dlo * grlo;
      if (lane + 32 < k) part += sd[lane + 32] * red.dhi * grhi;
      const T csum = bx_warp_sum(part);
      const T term2 = csq * rsq;  // |d|^2 |c|^2 |r|^2
      norm2 += T(2) * delta * csum + term2;
      small = (term2 <= tol2 * norm2) ? small + 1 : 0;
      if (k == 0) pfloor = fabs(delta) * (T)(sizeof(T) == 4 ? 1e-9 : 1e-20);
      if (q == 0 && warp == 0) {
        if (lane == 0) {
          B.GC[k + (size_t)k * p.kcap] = (double)csq;
          B.GR[k + (size_t)k * p.kcap] = (double)rr;
          B.d[k] = (double)delta;
          B.I[k] = istar;
          B.J[k] = jstar;
        }
        for (int h = 0; h < 2; ++h) {
          const int l = lane + 32 * h;
          if (l < k) {
            const double gc = (double)(h ? red.dhi : red.dlo), gr = (double)(h ? grhi : grlo);
            B.GC[l + (size_t)k * p.kcap] = gc;
            B.GC[k + (size_t)l * p.kcap] = gc;
            B.GR[l + (size_t)k * p.kcap] = gr;
            B.GR[k + (size_t)l * p.kcap] = gr;
          }
        }
      }
    }
    // the next row half-step needs column k of C: the winner's own value
    pv = {red.cand, k, inext >= 0 ? 1 : 0, red.val};
    ++k;
    if (small >= 2) {
      if (probe_rounds >= cp.max_probe_rounds || cp.probes <= 0) { converged = 1; break; }
      // residual probes at splitmix64-drawn entries; probe pr on warp pr mod
      // (warps per CTA), the same arithmetic in every CTA
      __syncthreads();  // sd[k - 1]
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
          sk += (double)__ldcg(&p.C[pi + (size_t)l * p.ld]) * (double)sd[l] *
                (double)__ldcg(&p.R[pj + (size_t)l * p.ld]);
        num = bx_warp_sum(num);
        sk = bx_warp_sum(sk);
        const double den = (double)p.a[pi] * (double)p.b[pj] + (double)p.b[pi] * (double)p.a[pj];
        if (lane == 0) { sprobe[pr] = fabs(num / den - sk); sprow[pr] = pi; }
      }
      // the probes read skeleton entries other CTAs wrote in this step
      if (cs > 1) cl.sync(); else __syncthreads();
      double worst = -1.0;
      int wrow = -1;
      for (int pr = 0; pr < Pn; ++pr)
        if (sprobe[pr] > worst) { worst = sprobe[pr]; wrow = sprow[pr]; }
      const double n2 = (double)norm2;
      ++probe_rounds;
      if (worst <= cp.tol * sqrt(n2 > 0.0 ? n2 : 0.0)) { converged = 1; break; }
      small = 0;
      // restart at the bad probe's row if unused, else at the best unused score
      bx_scores<T, RPT>(p, a0, b0, v);
      {
        const int s = slot(wrow);
        if (s >= 0 && !((used_r >> s) & 1u)) {
#pragma unroll
          for (int ss = 0; ss < RPT; ++ss)
            if (ss == s) v[ss] = T(INFINITY);
        }
      }
      red = bx_reduce<T, RPT>(p, v, own & ~used_r, p.C, 0, p.Uh, p.C, k, par);
      istar = red.idx;
      if (istar < 0) { converged = 1; break; }
      pv = {red.cand, k, 0, T(0)};
      continue;
    }
    istar = inext;
    if (istar < 0) { converged = 1; break; }
  }
  // no CTA may exit while another can still write into its shared memory
  if (cs > 1) cl.sync();
  if (q == 0 && tid == 0) {
    st->k = k;
    st->converged = converged;
    st->probe_rounds = probe_rounds;
    st->zero_rows = zero_rows;
    st->norm2 = (double)norm2;
  }
}

template <typename T, int RPT>
cudaError_t launch_bcross_rpt(const BatchProb* probs, const int* list, int n, int cs,
                              const BatchCrossParams& cp, cudaStream_t st) {
  auto kern = bcross_kernel<T, RPT>;
  const size_t smax = ((size_t)(2 * BX_NW + 2 * 16) * BX_WORDS + 2 * BX_RES) * sizeof(T);
  static cudaError_t attr = [&] {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * cs), 1, 1);
  cfg.blockDim = dim3(BX_NT, 1, 1);
  cfg.dynamicSmemBytes = ((size_t)(2 * BX_NW + 2 * cs) * BX_WORDS + 2 * BX_RES) * sizeof(T);
  cfg.stream = st;
  cudaLaunchAttribute attr_[1];
  attr_[0].id = cudaLaunchAttributeClusterDimension;
  attr_[0].val.clusterDim.x = cs;
  attr_[0].val.clusterDim.y = 1;
  attr_[0].val.clusterDim.z = 1;
  cfg.attrs = attr_;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, probs, list, cp);
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
