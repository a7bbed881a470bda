// In-place FFT stages for transforms that hold a whole sequence in one CTA's
// shared memory (the one-pass batched sine transform, batch.cu).
//
// Forward: decimation in frequency, natural order in, digit-reversed order
// out.  Inverse: its adjoint, decimation in time with conjugate twiddles,
// digit-reversed order in, natural order out, unnormalised.  A pointwise
// product with a spectrum stored in the same digit-reversed order between
// the two therefore needs no reordering, and every butterfly writes back to
// the positions it read: a stage needs one barrier and only one butterfly's
// values in registers (a Stockham pass holds the whole sequence in
// registers between its read and its write phase).
//
// Stages of a length-H sequence (H = 2^logH): n16 = logH / 4 radix-16 stages
// on blocks of length L = H, H/16, ... (span s = L/16: butterfly j < s of a
// block takes its elements j + q s, q < 16), then one radix-2^(logH mod 4)
// stage on blocks of 2 or 4 contiguous elements, whose twiddles are all 1.
// A radix-16 butterfly is two radix-4 layers: element u + 4v (u, v < 4)
//   layer A: for each u, 4-point DFT over v, output p times
//            w_L^((j + u s) p) = a_p w_16^(u p), a_p = w_L^(j p);
//   layer B: for each p, 4-point DFT over u, output p2 times
//            w_(4s)^(j p2) = b_p2, b_p2 = w_L^(4 j p2);
// result (p, p2) at element 4 p + p2.  Position -> frequency: inplace_freq.
#pragma once

#include "fft_common.cuh"

namespace lrp {

// Frequency held at digit-reversed position pos of a length-2^logH forward
// transform: digits of pos (most significant first; radix 4 for each layer
// of the radix-16 stages, then the last stage's radix) read least
// significant first.
__host__ __device__ inline long long inplace_freq(long long pos, int logH) {
  const int n16 = logH >> 2, rem = logH & 3;
  long long wgt = 1LL << logH, k = 0, mul = 1;
  for (int i = 0; i < 2 * n16; ++i) {
    wgt >>= 2;
    k += ((pos / wgt) & 3) * mul;
    mul <<= 2;
  }
  if (rem) {
    wgt >>= rem;
    k += ((pos / wgt) & ((1 << rem) - 1)) * mul;
  }
  return k;
}

// Twiddle tables of the radix-16 stages: stage i (L = H / 16^i, s = L / 16)
// holds six planes of s values, a_p(j) = w_L^(j p) and b_p(j) = w_L^(4 j p),
// p = 1..3, planes contiguous in j (consecutive lanes, consecutive words).
__host__ __device__ constexpr int inplace_tab_elems(int logH) {
  int n = 0;
  for (int l = logH; l >= 4; l -= 4) n += 6 << (l - 4);
  return n;
}
__device__ __forceinline__ int inplace_tab_offset(int logH, int stage) {
  int n = 0;
  for (int i = 0; i < stage; ++i) n += 6 << (logH - 4 * i - 4);
  return n;
}

// Fill the tables for length 2^logH from tw[q] = exp(-2 pi i q / 2^logM),
// logM >= logH.  The caller synchronises afterwards.
template <typename T>
__device__ void build_inplace_tables(cpx<T>* tab, const cpx<T>* __restrict__ tw, int logM, int logH) {
  int off = 0;
  for (int logL = logH; logL >= 4; logL -= 4) {
    const int logS = logL - 4, s = 1 << logS;
    for (int idx = threadIdx.x; idx < 6 * s; idx += blockDim.x) {
      const int c = idx >> logS, j = idx & (s - 1);
      const int x = c < 3 ? j * (c + 1) : 4 * j * (c - 2);
      tab[off + idx] = tw[(size_t)x << (logM - logL)];
    }
    off += 6 * s;
  }
}

template <typename T>
__device__ __forceinline__ void dif16(cpx<T> (&x)[16], const cpx<T> (&a)[3], const cpx<T> (&b)[3]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    dft4(x[u], x[u + 4], x[u + 8], x[u + 12], false);
#pragma unroll
    for (int p = 1; p < 4; ++p) {
      cpx<T> t = cmul(x[u + 4 * p], a[p - 1]);
      if (u > 0) t = cmul(t, w16<T>(u * p, false));
      x[u + 4 * p] = t;
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    dft4(x[4 * p], x[4 * p + 1], x[4 * p + 2], x[4 * p + 3], false);
#pragma unroll
    for (int p2 = 1; p2 < 4; ++p2) x[4 * p + p2] = cmul(x[4 * p + p2], b[p2 - 1]);
  }
}

// Adjoint of dif16 (conjugate twiddles, inverse 4-point DFTs, layers in
// reverse order).
template <typename T>
__device__ __forceinline__ void dit16(cpx<T> (&x)[16], const cpx<T> (&a)[3], const cpx<T> (&b)[3]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
#pragma unroll
    for (int p2 = 1; p2 < 4; ++p2) x[4 * p + p2] = cmulc(x[4 * p + p2], b[p2 - 1]);
    dft4(x[4 * p], x[4 * p + 1], x[4 * p + 2], x[4 * p + 3], true);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int p = 1; p < 4; ++p) {
      cpx<T> t = cmulc(x[u + 4 * p], a[p - 1]);
      if (u > 0) t = cmul(t, w16<T>(u * p, true));
      x[u + 4 * p] = t;
    }
    dft4(x[u], x[u + 4], x[u + 8], x[u + 12], true);
  }
}

// The twiddles of butterfly j of a stage (table of that stage, span s).
template <typename T>
__device__ __forceinline__ void stage_twiddles(const cpx<T>* tabi, int s, int j, cpx<T> (&a)[3], cpx<T> (&b)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a[c] = tabi[c * s + j];
    b[c] = tabi[(3 + c) * s + j];
  }
}

// Padded-index offset of element q s of a butterfly from its first element
// b (smem_ix<true>): q s + (q s) / 16 whenever b mod 16 < s or s is a
// multiple of 16, which holds for every butterfly of the stages below (b =
// B 16 s + j, j < s).  Constant per q and s, so every access of a butterfly
// is one shared-memory instruction with an immediate offset.
__host__ __device__ constexpr int pad_off(int qs) { return qs + (qs >> 4); }

// One radix-16 stage with compile-time sizes: 2^LOGN padded elements,
// span 2^LOGS, NT threads.
template <typename T, bool INV, int NT, int LOGN, int LOGS>
__device__ __forceinline__ void inplace_stage16c(cpx<T>* buf, const cpx<T>* tabi) {
  constexpr int nb = 1 << (LOGN - 4), s = 1 << LOGS;
#pragma unroll
  for (int g0 = 0; g0 < nb; g0 += NT) {
    const int g = g0 + (int)threadIdx.x;
    if (nb % NT != 0 && g >= nb) break;
    const int j = g & (s - 1);
    cpx<T>* bp = buf + smem_ix<true>(((g >> LOGS) << (LOGS + 4)) + j);
    cpx<T> x[16], a[3], b[3];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = bp[pad_off(q << LOGS)];
    stage_twiddles(tabi, s, j, a, b);
    if (INV) dit16(x, a, b);
    else dif16(x, a, b);
#pragma unroll
    for (int q = 0; q < 16; ++q) bp[pad_off(q << LOGS)] = x[q];
  }
}

// One radix-16 stage over a buffer of 2^logN padded elements (several
// sequences of length >= 16 s back to back), span s = 2^logS, NT threads.
template <typename T, bool INV, int NT>
__device__ __forceinline__ void inplace_stage16(cpx<T>* buf, int logN, int logS, const cpx<T>* tabi) {
  const int nb = 1 << (logN - 4), s = 1 << logS;
  for (int g = threadIdx.x; g < nb; g += NT) {
    const int j = g & (s - 1);
    const int base = ((g >> logS) << (logS + 4)) + j;
    cpx<T> x[16], a[3], b[3];
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = buf[smem_ix<true>(base + (q << logS))];
    stage_twiddles(tabi, s, j, a, b);
    if (INV) dit16(x, a, b);
    else dif16(x, a, b);
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[smem_ix<true>(base + (q << logS))] = x[q];
  }
}

// The last forward stage (RL = 2, 4 or 16 contiguous elements, twiddles 1),
// the product with the spectrum spec (digit-reversed order, length 2^logH,
// every sequence of the buffer), and the first inverse stage, in registers.
template <typename T, int RL, int NT, int N>
__device__ __forceinline__ void inplace_last(cpx<T>* buf, int logH, const cpx<T>* __restrict__ spec) {
  constexpr int NB = N / RL, NI = (NB + NT - 1) / NT;
  const int hmask = (1 << logH) - 1;
  // every spectrum value of the thread first: one global-memory wait
  cpx<T> sp[NI][RL];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int g = i * NT + (int)threadIdx.x;
#pragma unroll
    for (int q = 0; q < RL; ++q) sp[i][q] = g < NB ? spec[(g * RL + q) & hmask] : cpx<T>{T(0), T(0)};
  }
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int g = i * NT + (int)threadIdx.x;
    if (NB % NT != 0 && g >= NB) break;
    const int base = g * RL;
    cpx<T>* bp = buf + smem_ix<true>(base);  // RL contiguous elements, no pad inside
    cpx<T> x[RL];
#pragma unroll
    for (int q = 0; q < RL; ++q) x[q] = bp[q];
    if constexpr (RL == 16) {
      cpx<T> one[3] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
      dif16(x, one, one);
#pragma unroll
      for (int q = 0; q < RL; ++q) x[q] = cmul(x[q], sp[i][q]);
      dit16(x, one, one);
    } else if constexpr (RL == 4) {
      dft4(x[0], x[1], x[2], x[3], false);
#pragma unroll
      for (int q = 0; q < RL; ++q) x[q] = cmul(x[q], sp[i][q]);
      dft4(x[0], x[1], x[2], x[3], true);
    } else {
      cpx<T> y0 = cadd(x[0], x[1]), y1 = csub(x[0], x[1]);
      y0 = cmul(y0, sp[i][0]);
      y1 = cmul(y1, sp[i][1]);
      x[0] = cadd(y0, y1);
      x[1] = csub(y0, y1);
    }
#pragma unroll
    for (int q = 0; q < RL; ++q) bp[q] = x[q];
  }
}

}  // namespace lrp
