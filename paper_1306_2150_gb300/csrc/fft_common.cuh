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
    } else {
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
// bank.  Planes r = 1, 2, 3 in float32 (each value rounded once); float64
// keeps the r = 1 plane and forms w_2 = w_1^2, w_3 = w_1 w_2.
//   stw[(r - 1) kStageSize + 2^logNs - 1 + k],  logNs <= kStageLog.
// ---------------------------------------------------------------------------
constexpr int kStageLog = 10;                      // up to Ns = 1024: FFT lengths <= 4096
constexpr int kStageSize = (2 << kStageLog) - 1;   // entries per plane
template <typename T> __host__ __device__ constexpr int stage_planes() { return sizeof(T) == 4 ? 3 : 1; }
template <typename T> __host__ __device__ constexpr int stage_elems() { return stage_planes<T>() * kStageSize; }

// Fill the stages logNs <= maxLogNs from a full table tw[q] = exp(-2 pi i q /
// 2^logTab) (logTab >= maxLogNs + 2).  The caller synchronises afterwards.
template <typename T>
__device__ __forceinline__ void build_stage_twiddles(cpx<T>* stw, const cpx<T>* __restrict__ tw, int logTab,
                                                     int maxLogNs) {
  constexpr int P = stage_planes<T>();
  if (maxLogNs < 0) return;
  const int n = (2 << maxLogNs) - 1;
  for (int idx = threadIdx.x; idx < P * n; idx += blockDim.x) {
    const int rm1 = idx / n, e = idx - rm1 * n;
    const int logNs = 31 - __clz(e + 1);  // e in [2^logNs - 1, 2^(logNs+1) - 1)
    const int k = e + 1 - (1 << logNs);
    stw[rm1 * kStageSize + e] = tw[(size_t)((rm1 + 1) * k) << (logTab - 2 - logNs)];
  }
}

template <typename T, int LOGR, bool FMAJOR>
__device__ __forceinline__ void stockham_pass_st(cpx<T>* buf, int logL, int lognf, int es, int fs, int logNs,
                                                 const cpx<T>* __restrict__ stw, bool inverse) {
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
    for (int r = 0; r < R; ++r) x[r] = buf[f * fs + (j + (r << logLR)) * es];
    if (R == 4) {  // a radix-2 pass only runs at Ns = 1, where every twiddle is 1
      cpx<T> w1 = st1[k], w2, w3;
      if (stage_planes<T>() == 3) {
        w2 = st1[kStageSize + k];
        w3 = st1[2 * kStageSize + k];
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
    } else {
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

// Full length-2^logL FFT (logL <= kStageLog + 2) of 2^lognf sequences with
// the stage tables; blockDim.x * EPT must equal 2^(logL + lognf).
template <typename T, bool FMAJOR>
__device__ void smem_fft_st(cpx<T>* buf, int logL, int lognf, int es, int fs, const cpx<T>* __restrict__ stw,
                            bool inverse) {
  int logNs = 0;
  if (logL & 1) {
    stockham_pass_st<T, 1, FMAJOR>(buf, logL, lognf, es, fs, logNs, stw, inverse);
    logNs += 1;
  }
  while (logNs < logL) {
    stockham_pass_st<T, 2, FMAJOR>(buf, logL, lognf, es, fs, logNs, stw, inverse);
    logNs += 2;
  }
}

}  // namespace lrp
