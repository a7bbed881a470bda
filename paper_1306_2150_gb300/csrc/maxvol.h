// Internal interface of the maxvol row selection (maxvol.cu), called by
// lr_maxvol in api.cu.
#pragma once

#include <cuda_runtime.h>

namespace lrp {

// Device record of one selection.  Zeroed by the host before the first launch.
struct MvState {
  int i, j;             // row and column of the pending swap: rows[j] becomes i
  double piv;           // B[i, j] of that swap
  double bmax;          // largest |B| seen by the last decision
  int done;             // 1 once the selection stopped (dominant, swap cap or error)
  int nswaps;           // swaps decided so far
  int status;           // bit 0: C[rows, :] singular; bit 1: non-finite coefficient
  unsigned int ticket;  // last-CTA counter of the reduction (reset by the last CTA)
};

struct MvArgs {
  const double* C;      // m x k, column-major, leading dimension ldc
  int ldc, m, k;
  double delta;         // stop once every |B| <= 1 + delta
  int maxswaps;
  double* B;            // m x k coefficients C C[rows, :]^{-1}, leading dimension ldb
  int ldb;
  double* Ainv;         // MV_KMAX x MV_KMAX (row p, column l at p * MV_KMAX + l), zero padded
  double* row;          // MV_KMAX: B[i, :] of the pending swap
  double* pabs;         // grid: per-CTA largest |B|
  long long* pidx;      // grid: its column-major index j m + i
  int* rows;            // k selected rows (device)
  MvState* st;
  int grid;             // CTAs of the coefficient and swap kernels
};

constexpr int MV_KMAX = 64;
constexpr int MV_THREADS = 128;

int maxvol_grid(int m, int num_sms);
// Inverse of C[rows, :] (Gauss-Jordan with partial pivoting), B = C C[rows, :]^{-1}
// and the first decision.
cudaError_t launch_maxvol_start(const MvArgs& a, cudaStream_t st);
// One swap (B' = B - B[:, j] (B[i, :] - e_j^T) / B[i, j]) and the next decision;
// returns at once on the device when the selection has stopped.
cudaError_t launch_maxvol_swap(const MvArgs& a, cudaStream_t st);

}  // namespace lrp
