// DST-I of factor columns (Section 4.1: "DST of the factors U and V", the
// transform that diagonalises the Laplacian, Eq. flr:diag), on the GPU.
//
// The orthonormal DST-I of order m, y_k = sqrt(2/N) sum_j x_j sin(pi j k / N)
// (N = m + 1), is evaluated by Bluestein's chirp identity
//   j k = (j^2 + k^2 - (k - j)^2) / 2,  w_t = exp(i pi t^2 / (2N)),
//   y_k = sqrt(2/N) Im( w_k  sum_j (x_j w_j) conj(w_{k-j}) ),
// a linear convolution computed as a circular one of power-of-two length
// M >= 2m - 1 by FFT.  2N is not smooth for the grid sizes of interest
// (2 * 16385 = 2*5*29*113), so no mixed-radix FFT of length 2N is used.
//
// Kernels (complex working precision T = float or double):
//   small path (M <= 4096): one CTA holds whole sequences in shared memory:
//       chirp multiply, FFT, spectrum multiply, inverse FFT, chirp, store.
//   four-step path (M = M1 * M2): sequence index t = t1 + M1 t2,
//       frequency index k = k2 + M2 k1, scratch stored as [k2][t1]:
//     col_fwd : per t1, length-M2 FFT over t2, twiddle exp(-2 pi i t1 k2/M)
//     row_mid : per k2, length-M1 FFT over t1 -> k1, times the kernel
//               spectrum (stored in the same [k2][k1] order), inverse FFT,
//               twiddle exp(+2 pi i t1 k2/M)
//     col_inv : per t1, inverse length-M2 FFT over k2 -> t2, chirp, store.
//   The frequency-domain product is taken in the permuted order the forward
//   passes leave, so no transposition pass is needed.
//   cluster path (8192 <= M <= 131072, a variant the autotuner may pick):
//   one thread-block cluster per column holds the whole sequence in
//   distributed shared memory (see dst_cluster_kernel).  On GB300 it is
//   slower than the four-step path as measured (float64: its per-CTA work
//   lands on a few SMs' small FP64 units; float32: latency-bound at 8 warps
//   per CTA), so the four-step path is the default.
// Shared-memory FFTs are in-place Stockham radix-4 (one radix-2 pass when
// log2 L is odd): every thread keeps its 16 elements in registers between the
// read and the write phase of a pass.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "fft_common.cuh"
#include "fft_inplace.cuh"
#include "lr_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

// ---------------------------------------------------------------------------
// Column addressing.
// ---------------------------------------------------------------------------
struct ColArgs {
  const void* in[2];
  void* out[2];
  int ld_in[2];
  int ld_out[2];
  int ncol[2];
  const int* dyn_count;
  const void* tm[2];
  const int* k_dev;
  const void* sym_a;
  const void* sym_b;
};

enum : int { IN_F64 = 0, IN_WORK = 1, IN_ROT = 2, IN_DIV = 3 };

__device__ __forceinline__ bool col_live(const ColArgs& c, int col, int& seg, int& cc) {
  seg = col < c.ncol[0] ? 0 : 1;
  cc = seg ? col - c.ncol[0] : col;
  if (seg == 1 && cc >= c.ncol[1]) return false;
  if (c.dyn_count && cc >= *c.dyn_count) return false;
  return true;
}

// Element t of input column cc of segment seg.  IN_ROT: the column is the
// rotation sum_{l<k} X[t, l] Tm[l, cc] of a working-precision skeleton X.
template <typename T, int INM>
__device__ __forceinline__ T load_in(const ColArgs& c, int seg, int cc, int t) {
  if (INM == IN_F64) return (T)(static_cast<const double*>(c.in[seg])[(size_t)cc * c.ld_in[seg] + t]);
  if (INM == IN_WORK) return static_cast<const T*>(c.in[seg])[(size_t)cc * c.ld_in[seg] + t];
  if (INM == IN_DIV) {
    const T* a = static_cast<const T*>(c.sym_a);
    const T* b = static_cast<const T*>(c.sym_b);
    return static_cast<const T*>(c.in[seg])[(size_t)cc * c.ld_in[seg] + t] / (a[t] * b[cc] + b[t] * a[cc]);
  }
  const T* X = static_cast<const T*>(c.in[seg]);
  const T* tm = static_cast<const T*>(c.tm[seg]) + (size_t)cc * KMAX;
  const int k = *c.k_dev;
  const int ld = c.ld_in[seg];
  T acc = T(0);
  for (int l = 0; l < k; ++l) acc += X[(size_t)l * ld + t] * __ldg(&tm[l]);
  return acc;
}
template <typename T, bool OUT64>
__device__ __forceinline__ void store_out(const ColArgs& c, int seg, int cc, int t, T v) {
  if (OUT64) static_cast<double*>(c.out[seg])[(size_t)cc * c.ld_out[seg] + t] = (double)v;
  else static_cast<T*>(c.out[seg])[(size_t)cc * c.ld_out[seg] + t] = v;
}

struct GeomArgs {
  int m, logM, logM1, logM2;
  int ncols;        // total column slots (ncol0 + ncol1)
  int logTile;      // complex elements per four-step tile (2^logTile)
};

// ---------------------------------------------------------------------------
// Small path: 2^lognf sequences of length M per CTA.
// ---------------------------------------------------------------------------
template <typename T, int INM, bool OUT64>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) dst_small_kernel(
    ColArgs c, GeomArgs g, const cpx<T>* __restrict__ chirp, const cpx<T>* __restrict__ tw,
    const cpx<T>* __restrict__ bhat, int lognf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int M = 1 << g.logM;
  const int nf = 1 << lognf;
  const int items = (g.ncols + nf - 1) >> lognf;
  const int nelem = nf << g.logM;
  cpx<T>* stw = buf + nelem + (nelem >> 4);  // after the padded tile
  build_stage_twiddles(stw, tw, g.logM, g.logM - 2);
  const int stride = stage_stride(g.logM - 2);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    // Every loop below covers exactly EPT elements per thread; it is unrolled
    // so that a thread's global loads are all in flight together.
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        const int row = idx >> g.logM, t = idx & (M - 1);
        const int col = (item << lognf) + row;
        int seg, cc;
        v[s] = {T(0), T(0)};
        if (col < g.ncols && t < g.m && col_live(c, col, seg, cc)) {
          const T x = load_in<T, INM>(c, seg, cc, t);
          const cpx<T> w = chirp[t];
          v[s] = {x * w.re, x * w.im};
        }
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[smem_ix<true>(threadIdx.x + s * blockDim.x)] = v[s];
    }
    __syncthreads();
    smem_fft_st<T, false, true>(buf, g.logM, lognf, 1, M, stw, stride, false);
    {
      cpx<T> b[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) b[s] = bhat[(threadIdx.x + s * blockDim.x) & (M - 1)];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = smem_ix<true>(threadIdx.x + s * blockDim.x);
        buf[idx] = cmul(buf[idx], b[s]);
      }
    }
    __syncthreads();
    smem_fft_st<T, false, true>(buf, g.logM, lognf, 1, M, stw, stride, true);
#pragma unroll
    for (int s = 0; s < EPT; ++s) {
      const int idx = threadIdx.x + s * blockDim.x;
      const int row = idx >> g.logM, t = idx & (M - 1);
      const int col = (item << lognf) + row;
      int seg, cc;
      if (col < g.ncols && t < g.m && col_live(c, col, seg, cc)) {
        const cpx<T> w = chirp[t], z = buf[smem_ix<true>(idx)];
        store_out<T, OUT64>(c, seg, cc, t, w.re * z.im + w.im * z.re);  // Im(w z)
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Four-step path, column passes.  A tile holds TX = 4096 / M2 consecutive t1
// values and all M2 values of t2 (or k2): tile[t2 * TX + dt1].
// ---------------------------------------------------------------------------
template <typename T, int INM>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) dst_col_fwd_kernel(
    ColArgs c, GeomArgs g, const cpx<T>* __restrict__ chirp, const cpx<T>* __restrict__ tw,
    cpx<T>* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int M1 = 1 << g.logM1;
  const int tile = 1 << g.logTile;
  const int logTX = g.logTile - g.logM2, TX = 1 << logTX;
  const int blocks_per_col = M1 >> logTX;
  const int items = g.ncols * blocks_per_col;
  cpx<T>* stw = buf + tile;
  build_stage_twiddles(stw, tw, g.logM, g.logM2 - 2);
  const int stride = stage_stride(g.logM2 - 2);
  cpx<T>* th = stw + stage_elems<T>(std::max(g.logM1, g.logM2) - 2);  // inter-pass twiddles
  cpx<T>* tl = th + kTwHi;
  load_twiddles2(th, tl, tw, g.logM);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = item / blocks_per_col;
    const int t1_0 = (item - col * blocks_per_col) << logTX;
    int seg, cc;
    if (!col_live(c, col, seg, cc)) continue;  // uniform across the CTA
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        const int t2 = idx >> logTX, dt = idx & (TX - 1);
        const int t = t1_0 + dt + (t2 << g.logM1);
        v[s] = {T(0), T(0)};
        if (t < g.m) {
          const T x = load_in<T, INM>(c, seg, cc, t);
          const cpx<T> w = chirp[t];
          v[s] = {x * w.re, x * w.im};
        }
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[threadIdx.x + s * blockDim.x] = v[s];
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, g.logM2, logTX, TX, 1, stw, stride, false);
    cpx<T>* wc = work + ((size_t)col << g.logM);
    {
      cpx<T> w[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        w[s] = twiddle2(th, tl, (t1_0 + (idx & (TX - 1))) * (idx >> logTX));
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        const int k2 = idx >> logTX, t1 = t1_0 + (idx & (TX - 1));
        wc[(k2 << g.logM1) + t1] = cmul(buf[idx], w[s]);
      }
    }
    __syncthreads();
  }
}

template <typename T, bool OUT64>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) dst_col_inv_kernel(
    ColArgs c, GeomArgs g, const cpx<T>* __restrict__ chirp, const cpx<T>* __restrict__ tw,
    const cpx<T>* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int M1 = 1 << g.logM1;
  const int tile = 1 << g.logTile;
  const int logTX = g.logTile - g.logM2, TX = 1 << logTX;
  const int blocks_per_col = M1 >> logTX;
  const int items = g.ncols * blocks_per_col;
  cpx<T>* stw = buf + tile;
  build_stage_twiddles(stw, tw, g.logM, g.logM2 - 2);
  const int stride = stage_stride(g.logM2 - 2);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = item / blocks_per_col;
    const int t1_0 = (item - col * blocks_per_col) << logTX;
    int seg, cc;
    if (!col_live(c, col, seg, cc)) continue;
    const cpx<T>* wc = work + ((size_t)col << g.logM);
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        v[s] = wc[((idx >> logTX) << g.logM1) + t1_0 + (idx & (TX - 1))];
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) buf[threadIdx.x + s * blockDim.x] = v[s];
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, g.logM2, logTX, TX, 1, stw, stride, true);
#pragma unroll
    for (int s = 0; s < EPT; ++s) {
      const int idx = threadIdx.x + s * blockDim.x;
      const int t2 = idx >> logTX, dt = idx & (TX - 1);
      const int t = t1_0 + dt + (t2 << g.logM1);
      if (t < g.m) {
        const cpx<T> w = chirp[t], z = buf[idx];
        store_out<T, OUT64>(c, seg, cc, t, w.re * z.im + w.im * z.re);
      }
    }
    __syncthreads();
  }
}

// Row pass: RY = 4096 / M1 rows k2 per tile, each of M1 contiguous elements
// in global memory.  In shared memory the rows are interleaved, element e of
// row f at buf[e (RY + 1) + f], so that the FFT passes run with consecutive
// lanes on consecutive rows (no bank conflicts; the padding keeps the
// transposing loads and stores at two-way conflicts).
template <typename T>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 2 : 1) dst_row_mid_kernel(
    ColArgs c, GeomArgs g, const cpx<T>* __restrict__ tw, const cpx<T>* __restrict__ bhat,
    cpx<T>* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int M1 = 1 << g.logM1, M2 = 1 << g.logM2;
  const int tile = 1 << g.logTile;
  const int logRY = g.logTile - g.logM1;
  const int blocks_per_col = M2 >> logRY;
  const int items = g.ncols * blocks_per_col;
  const int RY = 1 << logRY, ES = RY + 1;
  cpx<T>* stw = buf + tile + M1;  // after the padded tile (M1 x (RY + 1))
  build_stage_twiddles(stw, tw, g.logM, g.logM1 - 2);
  const int stride = stage_stride(g.logM1 - 2);
  cpx<T>* th = stw + stage_elems<T>(std::max(g.logM1, g.logM2) - 2);  // inter-pass twiddles
  cpx<T>* tl = th + kTwHi;
  load_twiddles2(th, tl, tw, g.logM);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = item / blocks_per_col;
    const int k2_0 = (item - col * blocks_per_col) << logRY;
    int seg, cc;
    if (!col_live(c, col, seg, cc)) continue;
    cpx<T>* wc = work + ((size_t)col << g.logM) + ((size_t)k2_0 << g.logM1);
    const cpx<T>* bh = bhat + ((size_t)k2_0 << g.logM1);
    {
      cpx<T> v[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) v[s] = wc[threadIdx.x + s * blockDim.x];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        buf[(idx & (M1 - 1)) * ES + (idx >> g.logM1)] = v[s];
      }
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, g.logM1, logRY, ES, 1, stw, stride, false);
    {
      cpx<T> b[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) b[s] = bh[threadIdx.x + s * blockDim.x];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        const int bi = (idx & (M1 - 1)) * ES + (idx >> g.logM1);
        buf[bi] = cmul(buf[bi], b[s]);
      }
    }
    __syncthreads();
    smem_fft_st<T, true>(buf, g.logM1, logRY, ES, 1, stw, stride, true);
    {
      cpx<T> w[EPT];
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        w[s] = twiddle2(th, tl, (idx & (M1 - 1)) * (k2_0 + (idx >> g.logM1)));
      }
#pragma unroll
      for (int s = 0; s < EPT; ++s) {
        const int idx = threadIdx.x + s * blockDim.x;
        wc[idx] = cmulc(buf[(idx & (M1 - 1)) * ES + (idx >> g.logM1)], w[s]);  // times exp(+2 pi i t1 k2 / M)
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host launcher.
// ---------------------------------------------------------------------------
template <typename T>
static const TablesT& tables_of(const Plan& p);
template <> const TablesT& tables_of<double>(const Plan& p) { return p.t64; }
template <> const TablesT& tables_of<float>(const Plan& p) { return p.t32; }

// ---------------------------------------------------------------------------
// Cluster path (8192 <= M <= 131072): one thread-block cluster of CS = M / N2
// CTAs per column; CTA k1 ends up holding the length-N2 sub-spectrum k = k1 +
// CS k2 (N2 = 4096, or 8192 at M = 131072).  With t = t2 + N2 t1:
//   CTA c takes the t2 of its slice [c N2/CS, (c+1) N2/CS), reads a[t2 + N2 t1]
//   for every t1 from global memory, forms the CS-point DFTs in registers and
//   the twiddle, b_k1[t2] = w_M^(t2 k1) sum_t1 a[t2 + N2 t1] w_CS^(t1 k1), and
//   stores b_k1[t2] into CTA k1's shared memory (distributed shared memory);
//   CTA k1: A[k1 + CS k2] = FFT_N2(b_k1)[k2], times the kernel spectrum
//   (stored per CTA as [k1][k2]), d_k1 = conj(w_M^(t2 k1)) IFFT_N2(...);
//   CTA c again takes its slice, gathers d_k1[t2] from every CTA, forms the
//   inverse CS-point DFTs z[t2 + N2 t1] and stores Im(w_t z_t) for t < m.
// A transform is one launch, no scratch in global memory, inputs read and
// outputs written once (coalesced runs of N2/CS), and each value crosses the
// cluster network twice.
// ---------------------------------------------------------------------------
template <typename T, int INM, bool OUT64>
__global__ void __launch_bounds__(512) dst_cluster_kernel(ColArgs c, GeomArgs g, const cpx<T>* __restrict__ chirp,
                                                          const cpx<T>* __restrict__ tw,
                                                          const cpx<T>* __restrict__ bcl, int logN2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* S = reinterpret_cast<cpx<T>*>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int logCS = g.logM - logN2;
  const int me = (int)cl.block_rank();
  const int col = blockIdx.x >> logCS;
  const int NT = blockDim.x;        // N2 / EPT
  const int G = EPT >> logCS;       // slice positions per thread (EPT / CS)
  int seg, cc;
  const bool live = col < g.ncols && col_live(c, col, seg, cc);  // uniform over the cluster
  if (!live) return;
  const int slice0 = me << (logN2 - logCS);
  // Distributed shared memory may be written only once every CTA of the
  // cluster is running.
  cl.sync();
  // 1-2. a[t2 + N2 t1] of the slice from global memory, CS-point DFTs, twiddle,
  // scatter to the owners of the sub-spectra.
  for (int q = 0; q < G; ++q) {
    const int t2 = slice0 + threadIdx.x + q * NT;
    cpx<T> a[EPT];
#pragma unroll
    for (int t1 = 0; t1 < EPT; ++t1) {
      a[t1] = {T(0), T(0)};
      if (t1 < CS) {
        const int t = t2 + (t1 << logN2);
        if (t < g.m) {
          const T x = load_in<T, INM>(c, seg, cc, t);
          const cpx<T> w = chirp[t];
          a[t1] = {x * w.re, x * w.im};
        }
      }
    }
    for (int k1 = 0; k1 < CS; ++k1) {
      cpx<T> acc = a[0];
#pragma unroll
      for (int t1 = 1; t1 < EPT; ++t1)
        if (t1 < CS) acc = cadd(acc, cmul(a[t1], tw[((t1 * k1) & (CS - 1)) << logN2]));  // w_CS^(t1 k1)
      acc = cmul(acc, tw[(size_t)t2 * k1]);  // w_M^(t2 k1)
      cl.map_shared_rank(S, k1)[t2] = acc;
    }
  }
  cl.sync();
  // 3-5. local FFT, kernel spectrum, inverse FFT, conjugate twiddle
  smem_fft<T, false>(S, logN2, 0, 1, 0, tw, g.logM, false);
  {
    const cpx<T>* bk = bcl + ((size_t)me << logN2);
#pragma unroll
    for (int s = 0; s < EPT; ++s) {
      const int k2 = threadIdx.x + s * NT;
      S[k2] = cmul(S[k2], bk[k2]);
    }
  }
  __syncthreads();
  smem_fft<T, false>(S, logN2, 0, 1, 0, tw, g.logM, true);
#pragma unroll
  for (int s = 0; s < EPT; ++s) {
    const int t2 = threadIdx.x + s * NT;
    cpx<T> w = tw[(size_t)t2 * me];
    w.im = -w.im;
    S[t2] = cmul(S[t2], w);
  }
  cl.sync();
  // 6-7. gather the slice from every sub-spectrum owner, inverse CS-point
  // DFTs, chirp, store.
  for (int q = 0; q < G; ++q) {
    const int t2 = slice0 + threadIdx.x + q * NT;
    cpx<T> d[EPT];
#pragma unroll
    for (int k1 = 0; k1 < EPT; ++k1) d[k1] = k1 < CS ? cl.map_shared_rank(S, k1)[t2] : cpx<T>{T(0), T(0)};
    for (int t1 = 0; t1 < CS; ++t1) {
      const int t = t2 + (t1 << logN2);
      if (t >= g.m) break;  // t grows with t1
      cpx<T> z = d[0];
#pragma unroll
      for (int k1 = 1; k1 < EPT; ++k1)
        if (k1 < CS) {
          cpx<T> w = tw[((t1 * k1) & (CS - 1)) << logN2];
          w.im = -w.im;
          z = cadd(z, cmul(d[k1], w));
        }
      const cpx<T> w = chirp[t];
      store_out<T, OUT64>(c, seg, cc, t, w.re * z.im + w.im * z.re);  // Im(w z)
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T, int INM, bool OUT64>
static cudaError_t launch_dst_t(const Plan& p, const ColArgs& c, const GeomArgs& g, void* work,
                                int num_sms, cudaStream_t st) {
  const TablesT& tb = tables_of<T>(p);
  const cpx<T>* chirp = static_cast<const cpx<T>*>(tb.chirp);
  const cpx<T>* tw = static_cast<const cpx<T>*>(tb.tw);
  const cpx<T>* bhat = static_cast<const cpx<T>*>(tb.bhat);
  const int M = 1 << g.logM;
  if (M <= kSmallM) {
    // 2^lognf sequences per CTA so that every CTA has 4096 elements when
    // possible, but never more sequences than columns.
    // 2^lognf sequences per CTA: at least 512 elements (a warp of threads),
    // more only while there are still two CTAs per SM and the tile fits.
    int lognf = 0;
    while ((M << lognf) < 512) ++lognf;
    while ((M << (lognf + 1)) <= kTileElems && (g.ncols >> (lognf + 1)) >= 2 * num_sms) ++lognf;
    const int nelem = M << lognf;
    const int threads = nelem / EPT;
    const size_t smem = (size_t)(nelem + (nelem >> 4) + stage_elems<T>(g.logM - 2)) * sizeof(cpx<T>);
    const int items = (g.ncols + (1 << lognf) - 1) >> lognf;
    const int grid = items < 8 * num_sms ? items : 8 * num_sms;
    auto kern = dst_small_kernel<T, INM, OUT64>;
    static bool attr_set = false;  // once per instantiation: the largest tile plus the stage tables
    if (!attr_set) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (kTileElems + (kTileElems >> 4) + stage_elems<T>(kStageLog)) * (int)sizeof(cpx<T>));
      attr_set = true;
    }
    kern<<<grid, threads, smem, st>>>(c, g, chirp, tw, bhat, lognf);
    return cudaGetLastError();
  }
  // Cluster path: one cluster per column, no global scratch.
  if (p.logN2cl && p.use_cluster[sizeof(T) == 4 ? 1 : 0] &&
      (size_t)(1 << p.logN2cl) * sizeof(cpx<T>) <= 64 * 1024) {
    const int logN2 = p.logN2cl;
    const int CS = 1 << (g.logM - logN2);
    auto kern = dst_cluster_kernel<T, INM, OUT64>;
    const size_t smem = (size_t)(1 << logN2) * sizeof(cpx<T>);
    static cudaError_t attr = [&] {
      cudaError_t e1 = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
      return e1 != cudaSuccess ? e1 : e2;
    }();
    if (attr == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(g.ncols * CS));
      cfg.blockDim = dim3((unsigned)((1 << logN2) / EPT));
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = CS;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const cpx<T>* bcl = static_cast<const cpx<T>*>(tb.bhat_cl);
      cudaError_t e = cudaLaunchKernelEx(&cfg, kern, c, g, chirp, tw, bcl, logN2);
      if (e == cudaSuccess) return cudaSuccess;
      if (e != cudaErrorInvalidClusterSize && e != cudaErrorLaunchOutOfResources &&
          e != cudaErrorInvalidConfiguration)
        return e;
      cudaGetLastError();  // cluster does not fit: use the four-step path
    }
  }
  // Tile of 4096 elements, halved (down to 1024, and not below either
  // sub-length) while that still leaves fewer than two tiles per SM.
  GeomArgs g2 = g;
  g2.logTile = 12;
  const int logMin = g.logM1 > 10 ? g.logM1 : 10;
  const int tuned = p.log_tile[sizeof(T) == 4 ? 1 : 0];
  if (tuned) {
    g2.logTile = tuned < logMin ? logMin : (tuned > 12 ? 12 : tuned);
  } else {
    while (g2.logTile > logMin && (g.ncols << (g.logM - g2.logTile)) < 2 * num_sms) --g2.logTile;
  }
  const int tile = 1 << g2.logTile;
  const int threads = tile / EPT;
  const int slog = std::max(g.logM1, g.logM2) - 2;
  const size_t smem = (size_t)(tile + (1 << g.logM1) + stage_elems<T>(slog) + kTwHi + kTwLo) * sizeof(cpx<T>);
  const int items_col = g.ncols * ((1 << g.logM1) >> (g2.logTile - g.logM2));
  const int items_row = g.ncols * ((1 << g.logM2) >> (g2.logTile - g.logM1));
  const int cap = 8 * num_sms;
  cpx<T>* wk = static_cast<cpx<T>*>(work);
  auto k1 = dst_col_fwd_kernel<T, INM>;
  auto k2 = dst_row_mid_kernel<T>;
  auto k3 = dst_col_inv_kernel<T, OUT64>;
  static bool attr_set = false;  // once per instantiation: the largest tile plus the stage tables
  if (!attr_set) {
    // m <= 131072: M1, M2 <= 512 (row padding <= 512, stages up to Ns = 128)
    const int mx = (kTileElems + 512 + stage_elems<T>(7) + kTwHi + kTwLo) * (int)sizeof(cpx<T>);
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr_set = true;
  }
  k1<<<items_col < cap ? items_col : cap, threads, smem, st>>>(c, g2, chirp, tw, wk);
  k2<<<items_row < cap ? items_row : cap, threads, smem, st>>>(c, g2, tw, bhat, wk);
  k3<<<items_col < cap ? items_col : cap, threads, smem, st>>>(c, g2, chirp, tw, wk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dst(const Plan& p, const ColumnSet& cs, IoType in_t, IoType out_t, void* work,
                       int num_sms, cudaStream_t st) {
  ColArgs c;
  for (int s = 0; s < 2; ++s) {
    c.in[s] = cs.in[s];
    c.out[s] = cs.out[s];
    c.ld_in[s] = cs.ld_in[s];
    c.ld_out[s] = cs.ld_out[s];
    c.ncol[s] = cs.ncol[s];
  }
  c.dyn_count = cs.dyn_count;
  c.tm[0] = cs.tm[0];
  c.tm[1] = cs.tm[1];
  c.k_dev = cs.k_dev;
  c.sym_a = cs.sym_a;
  c.sym_b = cs.sym_b;
  GeomArgs g{p.m, p.logM, p.logM1, p.logM2, cs.ncol[0] + cs.ncol[1], 12};
  if (g.ncols == 0) return cudaSuccess;
  const bool o64 = out_t == IoType::F64;
  if (in_t == IoType::F64)
    return o64 ? launch_dst_t<T, IN_F64, true>(p, c, g, work, num_sms, st)
               : launch_dst_t<T, IN_F64, false>(p, c, g, work, num_sms, st);
  if (in_t == IoType::ROT) {
    if (!o64) return cudaErrorInvalidValue;
    return launch_dst_t<T, IN_ROT, true>(p, c, g, work, num_sms, st);
  }
  if (in_t == IoType::DIV) {
    if (o64) return cudaErrorInvalidValue;
    return launch_dst_t<T, IN_DIV, false>(p, c, g, work, num_sms, st);
  }
  return o64 ? launch_dst_t<T, IN_WORK, true>(p, c, g, work, num_sms, st)
             : launch_dst_t<T, IN_WORK, false>(p, c, g, work, num_sms, st);
}

template cudaError_t launch_dst<double>(const Plan&, const ColumnSet&, IoType, IoType, void*, int, cudaStream_t);
template cudaError_t launch_dst<float>(const Plan&, const ColumnSet&, IoType, IoType, void*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Tiled transpose (the full-grid solve transforms rows as columns of the
// transpose): 32 x 32 tiles through shared memory, padded against bank
// conflicts, coalesced on both sides.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ in, int ldi, int m, int n,
                                                        T* __restrict__ out, int ldo) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = i0 + threadIdx.x, j = j0 + r;
    if (i < m && j < n) tile[r][threadIdx.x] = in[i + (size_t)j * ldi];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = j0 + threadIdx.x, i = i0 + r;
    if (i < m && j < n) out[j + (size_t)i * ldo] = tile[threadIdx.x][r];
  }
}

template <typename T>
cudaError_t launch_transpose(const T* in, int ldi, int m, int n, T* out, int ldo, cudaStream_t st) {
  dim3 grid((m + 31) / 32, (n + 31) / 32), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(in, ldi, m, n, out, ldo);
  return cudaGetLastError();
}
template cudaError_t launch_transpose<float>(const float*, int, int, int, float*, int, cudaStream_t);
template cudaError_t launch_transpose<double>(const double*, int, int, int, double*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Plan tables (built once per order m on the host in float64, uploaded).
// ---------------------------------------------------------------------------

// exp(2 pi i q / L) for 0 <= q < L, L a multiple of 4.  q is reduced to the
// first quadrant in integers and the angle kept below pi/4, so the float64
// result is within about one ulp.
static std::complex<double> cis2pi(long long q, long long L) {
  const long long quarter = L / 4;
  q %= L;
  if (q < 0) q += L;
  const int p = (int)(q / quarter);
  const long long r = q - p * quarter;
  double c, s;
  if (2 * r <= quarter) {
    const double th = 2.0 * M_PI * (double)r / (double)L;
    c = std::cos(th);
    s = std::sin(th);
  } else {
    const double th = 2.0 * M_PI * (double)(quarter - r) / (double)L;
    c = std::sin(th);
    s = std::cos(th);
  }
  switch (p) {
    case 0: return {c, s};
    case 1: return {-s, c};
    case 2: return {-c, -s};
    default: return {s, -c};
  }
}

// In-place iterative radix-2 FFT of length 2^logn (forward, exp(-2 pi i/n)).
static void host_fft(std::vector<std::complex<double>>& a, int logn) {
  const size_t n = (size_t)1 << logn;
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t step = n / len;
    for (size_t i = 0; i < n; i += len)
      for (size_t j = 0; j < len / 2; ++j) {
        const std::complex<double> w = std::conj(cis2pi((long long)(j * step), (long long)n));
        const std::complex<double> u = a[i + j], v = a[i + j + len / 2] * w;
        a[i + j] = u + v;
        a[i + j + len / 2] = u - v;
      }
  }
}

Plan::~Plan() {
  for (void* q : allocations) cudaFree(q);
}

template <typename T>
static std::string upload(Plan& p, const std::vector<std::complex<double>>& v, void** dst) {
  std::vector<cpx<T>> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = {(T)v[i].real(), (T)v[i].imag()};
  void* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(cpx<T>)) != cudaSuccess) return "cudaMalloc of plan table failed";
  p.allocations.push_back(d);
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(cpx<T>), cudaMemcpyHostToDevice) != cudaSuccess)
    return "upload of plan table failed";
  *dst = d;
  return "";
}

template <typename T>
static std::string upload_real(Plan& p, const std::vector<double>& v, T** dst) {
  std::vector<T> h(v.begin(), v.end());
  void* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) return "cudaMalloc of symbol failed";
  p.allocations.push_back(d);
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return "upload of symbol failed";
  *dst = static_cast<T*>(d);
  return "";
}

std::string build_plan(int m, Plan& p) {
  p.m = m;
  const long long N = (long long)m + 1;
  int logM = ilog2(2LL * m - 1);
  if (logM < 6) logM = 6;
  p.logM = logM;
  p.logM1 = (logM + 1) / 2;
  p.logM2 = logM / 2;
  const size_t M = (size_t)1 << logM;
  // chirp w_{t+1} = exp(2 pi i (t+1)^2 / (4N))
  std::vector<std::complex<double>> chirp(m), tw(M), b(M, {0.0, 0.0});
  for (int t = 0; t < m; ++t) {
    const long long u = t + 1;
    chirp[t] = cis2pi((u * u) % (4 * N), 4 * N);
  }
  for (size_t q = 0; q < M; ++q) tw[q] = std::conj(cis2pi((long long)q, (long long)M));
  // kernel conj(w_d) at d mod M for |d| <= m-1 (w_0 = 1, w_{-d} = w_d)
  b[0] = {1.0, 0.0};
  for (int d = 1; d < m; ++d) {
    const std::complex<double> wd = std::conj(chirp[d - 1]);
    b[d] = wd;
    b[M - d] = wd;
  }
  host_fft(b, logM);
  const double scale = std::sqrt(2.0 / (double)N) / (double)M;
  for (auto& z : b) z *= scale;
  std::vector<std::complex<double>> bh(M);
  if (M <= (size_t)kSmallM) {
    bh = b;
  } else {
    const size_t M1 = (size_t)1 << p.logM1, M2 = (size_t)1 << p.logM2;
    for (size_t k2 = 0; k2 < M2; ++k2)
      for (size_t k1 = 0; k1 < M1; ++k1) bh[k2 * M1 + k1] = b[k2 + M2 * k1];
  }
  std::string e;
  if (!(e = upload<double>(p, chirp, &p.t64.chirp)).empty()) return e;
  if (!(e = upload<double>(p, tw, &p.t64.tw)).empty()) return e;
  if (!(e = upload<double>(p, bh, &p.t64.bhat)).empty()) return e;
  if (!(e = upload<float>(p, chirp, &p.t32.chirp)).empty()) return e;
  if (!(e = upload<float>(p, tw, &p.t32.tw)).empty()) return e;
  if (!(e = upload<float>(p, bh, &p.t32.bhat)).empty()) return e;
  // one-pass batched transform (float32): residue order
  if (logM > 12) {
    const int logH = std::min(logM, kFusedLogH32);
    const size_t H = (size_t)1 << logH, R = M >> logH;
    std::vector<std::complex<double>> br(M);
    for (size_t t = 0; t < R; ++t)
      for (size_t pos = 0; pos < H; ++pos) br[t * H + pos] = b[R * (size_t)inplace_freq((long long)pos, logH) + t];
    if (!(e = upload<float>(p, br, &p.t32.bhat_rs)).empty()) return e;
  }
  // cluster path: chunks of N2 = 4096 (8192 at M = 131072), spectrum stored
  // per CTA as [k1][k2] = b[k1 + CS k2]
  if (logM >= 13 && logM <= 17) {
    p.logN2cl = logM <= 16 ? 12 : 13;
    const size_t N2c = (size_t)1 << p.logN2cl, CSc = M / N2c;
    std::vector<std::complex<double>> bc(M);
    for (size_t k1 = 0; k1 < CSc; ++k1)
      for (size_t k2 = 0; k2 < N2c; ++k2) bc[k1 * N2c + k2] = b[k1 + CSc * k2];
    if (!(e = upload<double>(p, bc, &p.t64.bhat_cl)).empty()) return e;
    if (!(e = upload<float>(p, bc, &p.t32.bhat_cl)).empty()) return e;
  }
  // Symbol: lambda_i = 4 sin^2(i pi/(2N)), 4 - lambda_i = 4 cos^2(i pi/(2N)).
  std::vector<double> a5(m), b5(m, 1.0), as(m), bs(m);
  const double N2 = (double)N * (double)N;
  for (int i = 0; i < m; ++i) {
    const std::complex<double> z = cis2pi(i + 1, 4 * N);  // angle (i+1) pi / (2N)
    const double lam = 4.0 * z.imag() * z.imag();
    const double lamc = 4.0 * z.real() * z.real();
    a5[i] = lam * N2;             // mu_i = lambda_i / h^2
    as[i] = lam * N2 / 16.0;      // lambda_i / (16 h^2)
    bs[i] = lamc;
  }
  if (!(e = upload_real<double>(p, a5, &p.sym_a64[0])).empty()) return e;
  if (!(e = upload_real<double>(p, b5, &p.sym_b64[0])).empty()) return e;
  if (!(e = upload_real<double>(p, as, &p.sym_a64[1])).empty()) return e;
  if (!(e = upload_real<double>(p, bs, &p.sym_b64[1])).empty()) return e;
  if (!(e = upload_real<float>(p, a5, &p.sym_a32[0])).empty()) return e;
  if (!(e = upload_real<float>(p, b5, &p.sym_b32[0])).empty()) return e;
  if (!(e = upload_real<float>(p, as, &p.sym_a32[1])).empty()) return e;
  if (!(e = upload_real<float>(p, bs, &p.sym_b32[1])).empty()) return e;
  return "";
}

}  // namespace lrp
