// Kernels of the low-rank Uzawa solve of the 2D Stokes problem on
// semi-staggered grids (Section 2, Eq. flr:stprob; Section 5).
//
// In low-rank format the discrete gradient and divergence act on the factors
// with the (n-1) x n bidiagonal matrices G = E - Z and H = E + Z of Section 2:
//   B_x (U s V^T) = (G U s / 4h) (H V)^T,   B_y (U s V^T) = (H U s / 4h) (G V)^T,
//   B_x^T (W t Z^T) = (G^T W t / 4h) (H^T Z)^T, B_y^T ... = (H^T W t / 4h) (G^T Z)^T,
// so they keep the rank; sums of low-rank terms are rounded in float64.
#include "lr_internal.h"

namespace lrp {

// out[:, j] = scale * w_j * OP(in[:, j]), j < r (w null: ones).
//   OP_G, OP_H : length n -> n - 1,  (G x)_i = x_{i+1} - x_i, (H x)_i = x_{i+1} + x_i
//   OP_GT, OP_HT: length n - 1 -> n, (G^T y)_i = y_{i-1} - y_i, (H^T y)_i = y_{i-1} + y_i
//                 (y_{-1} = y_{n-1} = 0)
__global__ void gh_kernel(int op, int n, const double* __restrict__ in, int ldi, int r,
                          const double* __restrict__ w, double scale, double* __restrict__ out, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (j >= r) return;
  const double* x = in + (size_t)j * ldi;
  const double c = scale * (w ? w[j] : 1.0);
  const double sg = (op == OP_G || op == OP_GT) ? -1.0 : 1.0;
  if (op == OP_G || op == OP_H) {
    if (i >= n - 1) return;
    out[i + (size_t)j * ldo] = c * (x[i + 1] + sg * x[i]);
  } else {
    if (i >= n) return;
    const double lo = i >= 1 ? x[i - 1] : 0.0;
    const double hi = i <= n - 2 ? x[i] : 0.0;
    out[i + (size_t)j * ldo] = c * (lo + sg * hi);
  }
}

cudaError_t launch_gh(int op, int n, const double* in, int ldi, int r, const double* w, double scale,
                      double* out, int ldo, cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  dim3 grid((n + 255) / 256, r);
  gh_kernel<<<grid, 256, 0, st>>>(op, n, in, ldi, r, w, scale, out, ldo);
  return cudaGetLastError();
}

// C = X^T Y for tall float64 X (rows x kx) and Y (rows x ky): per-block
// partial products in a fixed order, then a deterministic sum over blocks.
constexpr int kXGramRows = 32;

__global__ void __launch_bounds__(256) xgram_partial_kernel(const double* __restrict__ X, int ldx,
                                                            const double* __restrict__ Y, int ldy, int rows,
                                                            int kx, int ky, double* __restrict__ partial) {
  __shared__ double tx[kXGramRows * KMAX];
  __shared__ double ty[kXGramRows * KMAX];
  const int r0 = blockIdx.x * kXGramRows;
  const int nr = min(kXGramRows, rows - r0);
  for (int idx = threadIdx.x; idx < kXGramRows * kx; idx += blockDim.x) {
    const int i = idx % kXGramRows, l = idx / kXGramRows;
    tx[l * kXGramRows + i] = i < nr ? X[(size_t)l * ldx + r0 + i] : 0.0;
  }
  for (int idx = threadIdx.x; idx < kXGramRows * ky; idx += blockDim.x) {
    const int i = idx % kXGramRows, l = idx / kXGramRows;
    ty[l * kXGramRows + i] = i < nr ? Y[(size_t)l * ldy + r0 + i] : 0.0;
  }
  __syncthreads();
  double* out = partial + (size_t)blockIdx.x * KMAX * KMAX;
  for (int idx = threadIdx.x; idx < kx * ky; idx += blockDim.x) {
    const int p = idx % kx, q = idx / kx;
    double acc = 0.0;
    for (int i = 0; i < nr; ++i) acc += tx[p * kXGramRows + i] * ty[q * kXGramRows + i];
    out[p + q * KMAX] = acc;
  }
}

__global__ void xgram_sum_kernel(const double* __restrict__ partial, int nblk, int kx, int ky,
                                 double* __restrict__ C) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < kx * ky; idx += gridDim.x * blockDim.x) {
    const int p = idx % kx, q = idx / kx;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += partial[(size_t)b * KMAX * KMAX + p + q * KMAX];
    C[p + (size_t)q * kx] = acc;
  }
}

cudaError_t launch_cross_gram(const double* X, int ldx, const double* Y, int ldy, int rows, int kx, int ky,
                              double* C, double* partial, cudaStream_t st) {
  if (kx <= 0 || ky <= 0) return cudaSuccess;
  const int nblk = (rows + kXGramRows - 1) / kXGramRows;
  xgram_partial_kernel<<<nblk, 256, 0, st>>>(X, ldx, Y, ldy, rows, kx, ky, partial);
  xgram_sum_kernel<<<(kx * ky + 255) / 256, 256, 0, st>>>(partial, nblk, kx, ky, C);
  return cudaGetLastError();
}

// out[j] = sum_i X[i, j], out[r + j] = sum_i (-1)^i X[i, j]  (j < r; one CTA
// per column, fixed reduction order): the products with the two kernel
// modes of the pressure (constant, checkerboard).
__global__ void __launch_bounds__(256) colsums_kernel(const double* __restrict__ X, int ld, int rows, int r,
                                                      double* __restrict__ out) {
  __shared__ double s1[256], s2[256];
  const int j = blockIdx.x;
  const double* x = X + (size_t)j * ld;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    a += x[i];
    b += (i & 1) ? -x[i] : x[i];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[j] = s1[0];
    out[r + j] = s2[0];
  }
}

// Columns for the kernel projection: e[:, 0] = 1, e[:, 1] = (-1)^i.
__global__ void kernel_modes_kernel(int rows, double* __restrict__ e, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  e[i] = 1.0;
  e[i + (size_t)ld] = (i & 1) ? -1.0 : 1.0;
}

cudaError_t launch_colsums(const double* X, int ld, int rows, int r, double* out, cudaStream_t st) {
  if (r <= 0) return cudaSuccess;
  colsums_kernel<<<r, 256, 0, st>>>(X, ld, rows, r, out);
  return cudaGetLastError();
}

cudaError_t launch_kernel_modes(int rows, double* e, int ld, cudaStream_t st) {
  kernel_modes_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, e, ld);
  return cudaGetLastError();
}

// dst[j] = coef * (src ? src[j] : 1), j < n.
__global__ void scale_copy_kernel(int n, const double* __restrict__ src, double coef, double* __restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = coef * (src ? src[j] : 1.0);
}

cudaError_t launch_scale_copy(int n, const double* src, double coef, double* dst, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scale_copy_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, src, coef, dst);
  return cudaGetLastError();
}

}  // namespace lrp
