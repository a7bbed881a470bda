// Shared device/host definitions of the low-rank Poisson library (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lrpoisson.h"

namespace lrp {

// Largest number of cross steps (skeleton columns) a solve may take, and the
// largest rank a right-hand side or a truncated matrix may have.  The small
// k x k cores are held in shared memory of one CTA, which bounds both.
constexpr int KMAX = 64;

// Complex number of the working precision, aligned for vector loads.
template <typename T> struct alignas(2 * sizeof(T)) cpx { T re, im; };

template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {  // a * conj(b)
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }

// State of one cross approximation, written by the cross kernel and read by
// the core, the rotation and the inverse transform (all on the device), and
// copied to pinned host memory at the end of a solve.
struct SolveState {
  int k;              // skeleton columns built by the cross
  int rank;           // rank kept by the rounding (R)
  int converged;      // 1 if the cross stop test passed, 0 if it hit its cap
  int cut;            // 1 if the kept rank was cut to the output capacity
  int probe_rounds;
  int zero_rows;
  int status;         // lr_status of the device part
  int pad;
  double norm2;       // ||skeleton||_F^2 estimate of the cross
  double sigma0;      // largest kept singular value
};

inline int ilog2(long long x) { int l = 0; while ((1LL << l) < x) ++l; return l; }

}  // namespace lrp
