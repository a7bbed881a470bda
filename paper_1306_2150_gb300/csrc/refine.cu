// Iterative refinement of a mixed-precision solve in float64.
//
// For X = U diag(s) V^T and the operator A X = c (P X Q + Q X P) of either
// kind (P = tridiag(-1, 2, -1); Q = I for the 5-point Laplacian and
// tridiag(1, 2, 1) for the semi-staggered one, Section 2 and Section 4.1;
// c = 1/h^2 or 1/(16 h^2)), the residual F - A X with F = UF VF^T is the
// low-rank matrix
//     [UF, -c P U s, -c Q U s] [VF, Q V, P V]^T,
// formed here exactly in float64 (tridiagonal products on the factors).
//
// Its factors are each of the size of F while the product is of the size of
// the error of X, so rounding it through Gram matrices (which resolve only
// sqrt(eps64) of a factor) would lose it.  It is rounded instead through a
// QR factorisation of each factor by shifted Cholesky QR (Cholesky QR steps
// on column-equilibrated Gram matrices, the first ones shifted: Fukaya,
// Kannan, Nakatsukasa, Zhang and Yamamoto, SIAM J. Sci. Comput. 42 (2020)).
// Two shifted and two plain steps give orthonormal Q and a backward-stable R
// for factors of condition up to about 1/eps64 (the residual's factors come
// close: P V is nearly in the span of V); only exactly zero columns are
// dropped.  The small core R_L R_R^T then goes to the SVD of the rounding
// core (Section 3).
#include <cfloat>

#include "lr_internal.h"

namespace lrp {

// (tridiag(off, diag, off) x)_i for column x of length m (zero outside).
__device__ __forceinline__ double tri(const double* x, int i, int m, double diag, double off) {
  double v = diag * x[i];
  if (i > 0) v += off * x[i - 1];
  if (i + 1 < m) v += off * x[i + 1];
  return v;
}

__global__ void residual_factors_kernel(int m, int r, int R, const double* __restrict__ UF,
                                        const double* __restrict__ VF, int ldf, const double* __restrict__ U,
                                        const double* __restrict__ s, const double* __restrict__ V, int ldx,
                                        double c, double qd, double qo, double* __restrict__ L,
                                        double* __restrict__ Rt, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;  // 0 .. r + 2R - 1
  if (i >= m) return;
  double lv, rv;
  if (col < r) {
    lv = UF[i + (size_t)col * ldf];
    rv = VF[i + (size_t)col * ldf];
  } else if (col < r + R) {
    const int q = col - r;
    const double* u = U + (size_t)q * ldx;
    const double* v = V + (size_t)q * ldx;
    lv = -c * s[q] * tri(u, i, m, 2.0, -1.0);
    rv = tri(v, i, m, qd, qo);
  } else {
    const int q = col - r - R;
    const double* u = U + (size_t)q * ldx;
    const double* v = V + (size_t)q * ldx;
    lv = -c * s[q] * tri(u, i, m, qd, qo);
    rv = tri(v, i, m, 2.0, -1.0);
  }
  L[i + (size_t)col * ldo] = lv;
  Rt[i + (size_t)col * ldo] = rv;
}

cudaError_t launch_residual_factors(int m, int r, int R, const double* UF, const double* VF, int ldf,
                                    const double* U, const double* s, const double* V, int ldx, int op,
                                    double* L, double* Rt, int ldo, cudaStream_t st) {
  const double h = 1.0 / (m + 1);
  const double c = op == 0 ? 1.0 / (h * h) : 1.0 / (16.0 * h * h);
  const double qd = op == 0 ? 1.0 : 2.0, qo = op == 0 ? 0.0 : 1.0;
  dim3 grid((m + 255) / 256, r + 2 * R);
  residual_factors_kernel<<<grid, 256, 0, st>>>(m, r, R, UF, VF, ldf, U, s, V, ldx, c, qd, qo, L, Rt, ldo);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One Cholesky QR step on two factors at once (blockIdx.x = side).  Input:
// G = X^T X (q x q, ld q).  With D = diag(G)^(-1/2) (0 for a zero column):
//   D G D + shift I = Rs^T Rs      (Cholesky; a pivot below floor marks the
//                                   column dependent: its row and column of
//                                   Rs are dropped)
//   T    = D Rs^-1                 (so that X T has orthonormal columns)
//   Racc <- (Rs D^-1) Racc         (Racc = Rs D^-1 on the first step)
// T and Racc are column-major with leading dimension KMAX; qout[side] = q
// (the column count the rotation kernel reads from the device).
// ---------------------------------------------------------------------------
constexpr int KP2 = KMAX + 1;

struct CholQrSmem {
  double A[KMAX * KP2];   // working matrix, then L = Rs^T (lower, row-major A[i*KP2+j])
  double V[KMAX * KP2];   // L^-1 (lower, row-major)
  double Ro[KMAX * KP2];  // previous Racc (row-major)
  double dsc[KMAX];
  double inv[KMAX];
  int live[KMAX];
};

__global__ void __launch_bounds__(256) cholqr_step_kernel(CholQrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CholQrSmem& S = *reinterpret_cast<CholQrSmem*>(smem_raw);
  const int side = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int q = a.q;
  const double* G = a.G[side];
  double* T = a.T[side];
  double* Racc = a.Racc[side];
  for (int j = tid; j < q; j += NT) {
    const double g = G[j + (size_t)j * q];
    const bool ok = g > 0.0 && isfinite(g);
    S.dsc[j] = ok ? 1.0 / sqrt(g) : 0.0;
    S.live[j] = ok ? 1 : 0;
  }
  __syncthreads();
  for (int idx = tid; idx < q * q; idx += NT) {
    const int i = idx / q, j = idx % q;
    double v = G[i + (size_t)j * q] * S.dsc[i] * S.dsc[j];
    if (i == j) v = S.live[i] ? 1.0 + a.shift : 0.0;  // exact unit diagonal after equilibration
    S.A[i * KP2 + j] = v;
    if (!a.first) S.Ro[i * KP2 + j] = Racc[i + (size_t)j * KMAX];
  }
  __syncthreads();
  // Right-looking Cholesky on the lower triangle.
  for (int j = 0; j < q; ++j) {
    if (tid == 0) {
      const double p = S.A[j * KP2 + j];
      const bool ok = S.live[j] && p > a.floor_rel;
      S.live[j] = ok ? 1 : 0;
      const double l = ok ? sqrt(p) : 0.0;
      S.A[j * KP2 + j] = l;
      S.inv[j] = ok ? 1.0 / l : 0.0;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < q; i += NT) S.A[i * KP2 + j] *= S.inv[j];
    __syncthreads();
    const int rem = q - j - 1;
    if (S.live[j])
      for (int w = tid; w < rem * rem; w += NT) {
        const int i = j + 1 + w / rem, l = j + 1 + w % rem;
        if (l <= i) S.A[i * KP2 + l] -= S.A[i * KP2 + j] * S.A[l * KP2 + j];
      }
    __syncthreads();
  }
  // V = L^-1 by forward substitution, one column per thread (dropped rows
  // and columns stay zero).
  for (int c = tid; c < q; c += NT) {
    for (int i = 0; i < c; ++i) S.V[i * KP2 + c] = 0.0;
    S.V[c * KP2 + c] = S.inv[c];
    for (int i = c + 1; i < q; ++i) {
      double acc = 0.0;
      if (S.live[i] && S.live[c])
        for (int l = c; l < i; ++l) acc += S.A[i * KP2 + l] * S.V[l * KP2 + c];
      S.V[i * KP2 + c] = -acc * S.inv[i];
    }
  }
  __syncthreads();
  // R_step = Rs D^-1 with Rs = L^T, in place over L (row-major Rstep[l][i]
  // at A[l * KP2 + i], l >= i: column l of R_step is row l of L over d_l).
  for (int idx = tid; idx < q * q; idx += NT) {
    const int l = idx / q, i = idx % q;
    if (i <= l) S.A[l * KP2 + i] = S.dsc[l] > 0.0 ? S.A[l * KP2 + i] * (1.0 / S.dsc[l]) : 0.0;
  }
  __syncthreads();
  // T = D Rs^-1 = D V^T;  Racc <- R_step Racc.
  for (int idx = tid; idx < KMAX * KMAX; idx += NT) {
    const int i = idx % KMAX, j = idx / KMAX;  // column-major position (i, j)
    double t = 0.0, rn = 0.0;
    if (i < q && j < q && i <= j) {
      t = S.dsc[i] * S.V[j * KP2 + i];
      if (a.first) {
        rn = S.A[j * KP2 + i];
      } else {
        for (int l = i; l <= j; ++l) rn += S.A[l * KP2 + i] * S.Ro[l * KP2 + j];
      }
    }
    T[idx] = t;
    Racc[idx] = rn;
  }
  if (tid == 0) a.qout[side] = q;
}

cudaError_t launch_cholqr_step(const CholQrArgs& a, cudaStream_t st) {
  const size_t sm = sizeof(CholQrSmem);
  static cudaError_t set =
      cudaFuncSetAttribute(cholqr_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (set != cudaSuccess) return set;
  cholqr_step_kernel<<<2, 256, sm, st>>>(a);
  return cudaGetLastError();
}

// U[:, j] *= s[j] (unit = 0) or s[j] / s[0] (unit = 1) for j < *K.  At unit
// scale the correction's float32 solve never meets values near the ends of
// its range.
__global__ void fold_weights_kernel(int m, const int* K, double* __restrict__ U, int ld,
                                    const double* __restrict__ s, int unit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= m || j >= *K) return;
  const double s0 = s[0];
  U[i + (size_t)j * ld] *= unit ? (s0 > 0.0 ? s[j] / s0 : 0.0) : s[j];
}

// w[j] *= s[0] for j < n (undo the unit scaling on the correction's weights).
__global__ void scale_weights_kernel(int n, double* __restrict__ w, const double* __restrict__ s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) w[j] *= s[0];
}

cudaError_t launch_fold_weights(int m, int kmax, const int* K, double* U, int ld, const double* s, bool unit,
                                cudaStream_t st) {
  dim3 grid((m + 255) / 256, kmax);
  fold_weights_kernel<<<grid, 256, 0, st>>>(m, K, U, ld, s, unit ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_scale_weights(int n, double* w, const double* s, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scale_weights_kernel<<<1, 64, 0, st>>>(n, w, s);
  return cudaGetLastError();
}

// Columns of the exponential-sum solve (Section 4.1, known approaches): for
// term q of the quadrature, L[:, off + q r + a] = w_q exp(-t_q mu_i) Uh[i, a],
// R[:, off + q r + a] = exp(-t_q mu_i) Vh[i, a].
__global__ void expsum_cols_kernel(int m, int r, const double* __restrict__ Uh, const double* __restrict__ Vh,
                                   int ldh, const double* __restrict__ mu, const double* __restrict__ t,
                                   const double* __restrict__ w, double* __restrict__ L, double* __restrict__ R,
                                   int ldo, int off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;  // q r + a
  if (i >= m) return;
  const int q = col / r, a = col % r;
  const double e = exp(-t[q] * mu[i]);
  L[i + (size_t)(off + col) * ldo] = w[q] * e * Uh[i + (size_t)a * ldh];
  R[i + (size_t)(off + col) * ldo] = e * Vh[i + (size_t)a * ldh];
}

cudaError_t launch_expsum_cols(int m, int r, int nterms, const double* Uh, const double* Vh, int ldh,
                               const double* mu, const double* t, const double* w, double* L, double* R, int ldo,
                               int off, cudaStream_t st) {
  if (nterms <= 0) return cudaSuccess;
  dim3 grid((m + 255) / 256, nterms * r);
  expsum_cols_kernel<<<grid, 256, 0, st>>>(m, r, Uh, Vh, ldh, mu, t, w, L, R, ldo, off);
  return cudaGetLastError();
}

}  // namespace lrp
