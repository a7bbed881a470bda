// Shared-memory FFT building blocks of the sine transforms (dst.cu, batch.cu):
// in-place Stockham radix-4 passes (one radix-2 pass when log2 L is odd) with
// every thread keeping its EPT elements in registers between the read and the
// write phase of a pass.
#pragma once

#include "lr_common.cuh"

namespace lrp {

constexpr int EPT = 16;  // elements per thread in every FFT tile

// ---------------------------------------------------------------------------
// Shared-memory Stockham passes.  Element e of sequence f is buf[f*fs + e*es].
// FMAJOR: consecutive threads take consecutive sequences (column tiles, fs=1);
// otherwise consecutive threads take consecutive elements of one sequence.
// tw[q] = exp(-2 pi i q / M) with M = 2^logM >= L.
// ---------------------------------------------------------------------------
template <typename T, int LOGR, bool FMAJOR>
__device__ __forceinline__ void stockham_pass(cpx<T>* buf, int logL, int lognf, int es, int fs,
                                              int logNs, const cpx<T>* __restrict__ tw, int logM,
                                              bool inverse) {
  constexpr int R = 1 << LOGR;
  constexpr int NB = EPT / R;  // butterflies per thread
  const int NT = blockDim.x;
  const int logLR = logL - LOGR;
  const int maskLR = (1 << logLR) - 1;
  const int maskNs = (1 << logNs) - 1;
  const int twshift = logM - LOGR - logNs;
  cpx<T> v[EPT];
#pragma unroll
  for (int s = 0; s < NB; ++s) {
    const int g = threadIdx.x + s * NT;
    int f, j;
    if (FMAJOR) { f = g & ((1 << lognf) - 1); j = g >> lognf; }
    else { f = g >> logLR; j = g & maskLR; }
    const int k = j & maskNs;
    cpx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = buf[f * fs + (j + (r << logLR)) * es];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cpx<T> w = tw[(r * k) << twshift];
      if (inverse) w.im = -w.im;
      x[r] = cmul(x[r], w);
    }
    if (R == 2) {
      v[s * R + 0] = cadd(x[0], x[1]);
      v[s * R + 1] = csub(x[0], x[1]);
    } else if (R == 4) {
      const cpx<T> s0 = cadd(x[0], x[2]), s1 = csub(x[0], x[2]);
      const cpx<T> s2 = cadd(x[1], x[3]), s3 = csub(x[1], x[3]);
      // forward: X1 = s1 - i s3, X3 = s1 + i s3; inverse swaps them
      const cpx<T> mis3 = {s3.im, -s3.re};  // -i * s3
      v[s * R + 0] = cadd(s0, s2);
      v[s * R + 2] = csub(s0, s2);
      v[s * R + 1] = inverse ? csub(s1, mis3) : cadd(s1, mis3);
      v[s * R + 3] = inverse ? cadd(s1, mis3) : csub(s1, mis3);
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NB; ++s) {
    const int g = threadIdx.x + s * NT;
    int f, j;
    if (FMAJOR) { f = g & ((1 << lognf) - 1); j = g >> lognf; }
    else { f = g >> logLR; j = g & maskLR; }
    const int k = j & maskNs;
    const int base = ((j >> logNs) << (logNs + LOGR)) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[f * fs + (base + (r << logNs)) * es] = v[s * R + r];
  }
  __syncthreads();
}

// Full length-2^logL FFT of 2^lognf sequences; blockDim.x * EPT must equal
// the number of elements 2^(logL + lognf).  Unnormalised.
template <typename T, bool FMAJOR>
__device__ void smem_fft(cpx<T>* buf, int logL, int lognf, int es, int fs,
                         const cpx<T>* __restrict__ tw, int logM, bool inverse) {
  int logNs = 0;
  if (logL & 1) {
    stockham_pass<T, 1, FMAJOR>(buf, logL, lognf, es, fs, logNs, tw, logM, inverse);
    logNs += 1;
  }
  while (logNs < logL) {
    stockham_pass<T, 2, FMAJOR>(buf, logL, lognf, es, fs, logNs, tw, logM, inverse);
    logNs += 2;
  }
}

// Twiddles of a length-2^logL FFT, exp(-2 pi i j / L), copied into shared
// memory from the length-M table (tw[j * M / L]).
template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* twS, const cpx<T>* __restrict__ tw, int logL, int logM) {
  for (int j = threadIdx.x; j < (1 << logL); j += blockDim.x) twS[j] = tw[(size_t)j << (logM - logL)];
}

// ---------------------------------------------------------------------------
// Stage twiddle tables.  A radix-4 Stockham pass at sub-length Ns = 2^logNs
// multiplies element r of a butterfly with w_r(k) = exp(-2 pi i r k / (4 Ns)),
// k = j mod Ns; these values depend on Ns only, not on the transform length.
// Stored stage by stage, k contiguous, consecutive lanes (consecutive k) read
// consecutive words: no shared-memory bank conflicts, where indexing one
// full-length table with a stage-dependent stride made up to 32 lanes hit one
// bank.  Planes r = 1, 2, 3, each value rounded once (forming w_2, w_3 from
// w_1 would cost float32 accuracy, and float64 multiplies, which GB300 runs
// at a small fraction of its float32 rate).
//   stw[(r - 1) stride + 2^logNs - 1 + k],  logNs <= maxLogNs,
//   stride = stage_stride(maxLogNs) = 2^(maxLogNs + 1) - 1.
// An FFT of length 2^logL needs maxLogNs = logL - 2.
// ---------------------------------------------------------------------------
constexpr int kStageLog = 10;  // up to Ns = 1024: FFT lengths <= 4096
__host__ __device__ constexpr int stage_stride(int maxLogNs) { return maxLogNs < 0 ? 0 : (2 << maxLogNs) - 1; }
template <typename T> __host__ __device__ constexpr int stage_planes() { return 3; }
template <typename T> __host__ __device__ constexpr int stage_elems(int maxLogNs) {
  return stage_planes<T>() * stage_stride(maxLogNs);
}

// Fill the stages logNs <= maxLogNs from a full table tw[q] = exp(-2 pi i q /
// 2^logTab) (logTab >= maxLogNs + 2).  The caller synchronises afterwards.
template <typename T>
__device__ __forceinline__ void build_stage_twiddles(cpx<T>* stw, const cpx<T>* __restrict__ tw, int logTab,
                                                     int maxLogNs) {
  constexpr int P = stage_planes<T>();
  if (maxLogNs < 0) return;
  const int n = stage_stride(maxLogNs);
  for (int idx = threadIdx.x; idx < P * n; idx += blockDim.x) {
    const int rm1 = idx / n, e = idx - rm1 * n;
    const int logNs = 31 - __clz(e + 1);  // e in [2^logNs - 1, 2^(logNs+1) - 1)
    const int k = e + 1 - (1 << logNs);
    stw[idx] = tw[(size_t)((rm1 + 1) * k) << (logTab - 2 - logNs)];
  }
}

// Shared-memory index of element a with one pad word pair every 16 elements
// (PAD): spreads the strided accesses of the early passes of a single long
// sequence over the banks.
template <bool PAD>
__device__ __forceinline__ int smem_ix(int a) { return PAD ? a + (a >> 4) : a; }

// The three stage twiddles w_r(k), r = 1..3, of sub-length 2^logNs.
template <typename T>
__device__ __forceinline__ void stage_tw3(const cpx<T>* __restrict__ stw, int stride, int logNs, int k, bool inverse,
                                          cpx<T>& w1, cpx<T>& w2, cpx<T>& w3) {
  const cpx<T>* st = stw + (1 << logNs) - 1;
  w1 = st[k];
  if (stage_planes<T>() == 3) {
    w2 = st[stride + k];
    w3 = st[2 * stride + k];
  } else {
    w2 = cmul(w1, w1);
    w3 = cmul(w2, w1);
  }
  if (inverse) { w1.im = -w1.im; w2.im = -w2.im; w3.im = -w3.im; }
}

// Four-point DFT in place (forward: exp(-2 pi i/4) = -i; inverse: +i).
template <typename T>
__device__ __forceinline__ void dft4(cpx<T>& x0, cpx<T>& x1, cpx<T>& x2, cpx<T>& x3, bool inverse) {
  const cpx<T> s0 = cadd(x0, x2), s1 = csub(x0, x2);
  const cpx<T> s2 = cadd(x1, x3), s3 = csub(x1, x3);
  const cpx<T> mis3 = {s3.im, -s3.re};  // -i * s3
  x0 = cadd(s0, s2);
  x2 = csub(s0, s2);
  x1 = inverse ? csub(s1, mis3) : cadd(s1, mis3);
  x3 = inverse ? cadd(s1, mis3) : csub(s1, mis3);
}

// exp(-2 pi i e / 16) (conjugated for the inverse) for the exponents e = r1 q1
// of a radix-16 butterfly: cos and sin of multiples of pi/8.
template <typename T>
__device__ __forceinline__ cpx<T> w16(int e, bool inverse) {
  constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
  constexpr double s1 = 0.38268343236508977173;  // sin(pi/8)
  constexpr double h = 0.70710678118654752440;   // sqrt(2)/2
  double re, im;
  switch (e) {
    case 0: re = 1.0; im = 0.0; break;
    case 1: re = c1; im = -s1; break;
    case 2: re = h; im = -h; break;
    case 3: re = s1; im = -c1; break;
    case 4: re = 0.0; im = -1.0; break;
    case 6: re = -h; im = -h; break;
    default: re = -c1; im = s1; break;  // e = 9
  }
  return {(T)re, (T)(inverse ? -im : im)};
}

template <typename T, int LOGR, bool FMAJOR, bool PAD>
__device__ __forceinline__ void stockham_pass_st(cpx<T>* buf, int logL, int lognf, int es, int fs, int logNs,
                                                 const cpx<T>* __restrict__ stw, int stride, bool inverse) {
  constexpr int R = 1 << LOGR;
  constexpr int NB = EPT / R;  // butterflies per thread
  const int NT = blockDim.x;
  const int logLR = logL - LOGR;
  const int maskLR = (1 << logLR) - 1;
  const int maskNs = (1 << logNs) - 1;
  const cpx<T>* st1 = stw + (1 << logNs) - 1;
  cpx<T> v[EPT];
#pragma unroll
  for (int s = 0; s < NB; ++s) {
    const int g = threadIdx.x + s * NT;
    int f, j;
    if (FMAJOR) { f = g & ((1 << lognf) - 1); j = g >> lognf; }
    else { f = g >> logLR; j = g & maskLR; }
    const int k = j & maskNs;
    cpx<T> x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = buf[smem_ix<PAD>(f * fs + (j + (r << logLR)) * es)];
    if (R == 16) {
      // element r = r1 + 4 r2 carries w^(r k), w = exp(-2 pi i / (16 Ns)):
      // w^(4 r2 k) is the radix-4 stage twiddle of sub-length Ns, w^(r1 k)
      // the one of sub-length 4 Ns.  Four DFTs over r2, twiddles
      // w^(r1 k) exp(-2 pi i r1 q1 / 16), four DFTs over r1; output q1 + 4 q2.
      cpx<T> a1, a2, a3, b1, b2, b3;
      stage_tw3(stw, stride, logNs, k, inverse, a1, a2, a3);
      stage_tw3(stw, stride, logNs + 2, k, inverse, b1, b2, b3);
#pragma unroll
      for (int r1 = 0; r1 < 4; ++r1) {
        x[r1 + 4] = cmul(x[r1 + 4], a1);
        x[r1 + 8] = cmul(x[r1 + 8], a2);
        x[r1 + 12] = cmul(x[r1 + 12], a3);
        dft4(x[r1], x[r1 + 4], x[r1 + 8], x[r1 + 12], inverse);  // x[r1 + 4 q1] = Y[r1][q1]
      }
#pragma unroll
      for (int r1 = 1; r1 < 4; ++r1) {
        const cpx<T> b = r1 == 1 ? b1 : (r1 == 2 ? b2 : b3);
#pragma unroll
        for (int q1 = 0; q1 < 4; ++q1) {
          cpx<T> y = cmul(x[r1 + 4 * q1], b);
          if (q1 > 0) y = cmul(y, w16<T>(r1 * q1, inverse));
          x[r1 + 4 * q1] = y;
        }
      }
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1) {
        cpx<T> y0 = x[4 * q1], y1 = x[1 + 4 * q1], y2 = x[2 + 4 * q1], y3 = x[3 + 4 * q1];
        dft4(y0, y1, y2, y3, inverse);
        v[s * R + q1] = y0;  // q = q1 + 4 q2
        v[s * R + q1 + 4] = y1;
        v[s * R + q1 + 8] = y2;
        v[s * R + q1 + 12] = y3;
      }
    }
    if (R == 4) {  // a radix-2 pass only runs at Ns = 1, where every twiddle is 1
      cpx<T> w1 = st1[k], w2, w3;
      if (stage_planes<T>() == 3) {
        w2 = st1[stride + k];
        w3 = st1[2 * stride + k];
      } else {
        w2 = cmul(w1, w1);
        w3 = cmul(w2, w1);
      }
      if (inverse) { w1.im = -w1.im; w2.im = -w2.im; w3.im = -w3.im; }
      x[1] = cmul(x[1], w1);
      x[2] = cmul(x[2], w2);
      x[3] = cmul(x[3], w3);
    }
    if (R == 2) {
      v[s * R + 0] = cadd(x[0], x[1]);
      v[s * R + 1] = csub(x[0], x[1]);
    } else if (R == 4) {
      const cpx<T> s0 = cadd(x[0], x[2]), s1 = csub(x[0], x[2]);
      const cpx<T> s2 = cadd(x[1], x[3]), s3 = csub(x[1], x[3]);
      // forward: X1 = s1 - i s3, X3 = s1 + i s3; inverse swaps them
      const cpx<T> mis3 = {s3.im, -s3.re};  // -i * s3
      v[s * R + 0] = cadd(s0, s2);
      v[s * R + 2] = csub(s0, s2);
      v[s * R + 1] = inverse ? csub(s1, mis3) : cadd(s1, mis3);
      v[s * R + 3] = inverse ? cadd(s1, mis3) : csub(s1, mis3);
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NB; ++s) {
    const int g = threadIdx.x + s * NT;
    int f, j;
    if (FMAJOR) { f = g & ((1 << lognf) - 1); j = g >> lognf; }
    else { f = g >> logLR; j = g & maskLR; }
    const int k = j & maskNs;
    const int base = ((j >> logNs) << (logNs + LOGR)) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[smem_ix<PAD>(f * fs + (base + (r << logNs)) * es)] = v[s * R + r];
  }
  __syncthreads();
}

// Full length-2^logL FFT (logL <= kStageLog + 2) of 2^lognf sequences with
// the stage tables (built for at least logL - 2); blockDim.x * EPT must equal
// 2^(logL + lognf).
// float32: radix-16 passes (two radix-4 stages per trip through shared
// memory) after at most one radix-2 and one radix-4 pass; float64 keeps
// radix-4 passes (sixteen complex doubles per thread would not fit the
// register budget).
template <typename T, bool FMAJOR, bool PAD = false>
__device__ void smem_fft_st(cpx<T>* buf, int logL, int lognf, int es, int fs, const cpx<T>* __restrict__ stw,
                            int stride, bool inverse) {
  int logNs = 0;
  if (logL & 1) {
    stockham_pass_st<T, 1, FMAJOR, PAD>(buf, logL, lognf, es, fs, logNs, stw, stride, inverse);
    logNs += 1;
  }
  if constexpr (sizeof(T) == 4) {
    if ((logL - logNs) & 2) {
      stockham_pass_st<T, 2, FMAJOR, PAD>(buf, logL, lognf, es, fs, logNs, stw, stride, inverse);
      logNs += 2;
    }
    while (logNs < logL) {
      stockham_pass_st<T, 4, FMAJOR, PAD>(buf, logL, lognf, es, fs, logNs, stw, stride, inverse);
      logNs += 4;
    }
  } else {
    while (logNs < logL) {
      stockham_pass_st<T, 2, FMAJOR, PAD>(buf, logL, lognf, es, fs, logNs, stw, stride, inverse);
      logNs += 2;
    }
  }
}

// ---------------------------------------------------------------------------
// Inter-pass twiddles of a four-step FFT, exp(-2 pi i q / M) for 0 <= q < M
// (256 <= M <= 2^17), from two small shared tables instead of scattered
// loads from the length-M table: th[q >> 8] = exp(-2 pi i (q - q mod 256)/M),
// tl[q mod 256] = exp(-2 pi i (q mod 256) / M), w = th * tl.
// ---------------------------------------------------------------------------
constexpr int kTwHi = 512, kTwLo = 256;

// Load th, tl for M = 2^logM from the length-M table (the caller synchronises).
template <typename T>
__device__ __forceinline__ void load_twiddles2(cpx<T>* th, cpx<T>* tl, const cpx<T>* __restrict__ tw, int logM) {
  const int nh = 1 << (logM - 8);
  for (int i = threadIdx.x; i < nh + kTwLo; i += blockDim.x) {
    if (i < nh) th[i] = tw[(size_t)i << 8];
    else tl[i - nh] = tw[i - nh];
  }
}
template <typename T>
__device__ __forceinline__ cpx<T> twiddle2(const cpx<T>* th, const cpx<T>* tl, int q) {
  return cmul(th[q >> 8], tl[q & (kTwLo - 1)]);
}

}  // namespace lrp
