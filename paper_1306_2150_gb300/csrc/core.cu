// Rounding of a low-rank matrix (Section 3: "rounding" without a full SVD,
// O((n+m) r^2 + r^3)): for X = L diag(d) R^T with tall L, R (k columns),
//   L = Q_L Lc^T, R = Q_R Lr^T     (Lc, Lr lower-triangular Cholesky factors
//                                   of the Gram matrices L^T L, R^T R)
//   M = Lc^T diag(d) Lr = W S Z^T   (k x k core, one-sided Jacobi SVD)
//   keep the largest K singular values with sqrt(sum dropped s^2) <= eps ||s||
//   X ~= (L Tc) diag(s_K) (R Tr)^T,  Tc = Lc^-T W_K,  Tr = Lr^-T Z_K,
// so L Tc and R Tr have orthonormal columns.  The Gram matrices of the cross
// skeleton come for free from the cross (its norm update needs them); for
// lr_truncate they are formed by a tall-skinny reduction.
//
// The k x k work runs in one CTA.  GB300 executes FP64 at a small fraction of
// its FP32 rate, so the O(k^3 * sweeps) Jacobi iteration may run in FP32
// (mixed precision) while Cholesky, the core product and the triangular
// solves stay in FP64.
#include <cfloat>

#include "lr_internal.h"

namespace lrp {

constexpr int KP = KMAX + 1;  // padded row length of the shared k x k arrays

template <typename JT>
struct CoreSmem {
  double Lc[KMAX * KP];
  double Lr[KMAX * KP];
  JT Mx[KMAX * KP];   // column q at Mx[q * KP + i]
  JT Zm[KMAX * KP];
  double sig[KMAX];
  double g0c[KMAX], g0r[KMAX];
  double invc[KMAX], invr[KMAX];  // reciprocal Cholesky pivots
  double d[KMAX];
  int perm[KMAX];
  int flag;
  int K;
  // float64 cores only: float32 copies of the core and its rotations, then
  // an orthogonalised rotation and a product temporary (re-basing steps)
  double scrA[sizeof(JT) == 8 ? KMAX * KP : 1];
  double scrB[sizeof(JT) == 8 ? KMAX * KP : 1];
  double amax;
  double scale;  // power of two applied to M before the Jacobi iteration
  double red[3][8];  // per-warp partials (fixed summation order)
};

template <typename JT>
__device__ __forceinline__ JT warp_sum_t(JT v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Maximum of non-negative doubles: their bit patterns order like integers.
__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

template <typename JT> __device__ __forceinline__ JT rsqrt_t(JT x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <typename JT> __device__ __forceinline__ JT fdiv_t(JT a, JT b);
template <> __device__ __forceinline__ float fdiv_t<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv_t<double>(double a, double b) { return a / b; }


// Sweeps of one-sided (Hestenes) Jacobi with round-robin pair ordering on
// the ke columns of X (column c at X[c * KP + i], ke rows), accumulating the
// rotations in Z, until a sweep rotates nothing (at most max_sweeps).  One
// warp per pair: lanes hold rows (ke <= 64: two per lane) of both columns in
// registers for the inner products and the update.
// A pair is left alone when it is orthogonal to tol: the rounding error of
// the computed inner product itself is about k ulps, so a tighter test would
// rotate rounding noise forever.  Whatever the sweep count, the discarded
// columns' norms are exactly the error of the truncated product, because
// every rotation is orthogonal.
template <typename JT>
__device__ void jacobi_sweeps(JT* X, JT* Z, int ke, JT tol, int max_sweeps,
                              const unsigned char (*pc0)[KMAX / 2], const unsigned char (*pc1)[KMAX / 2],
                              int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
  const int npairs = ke / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < ke - 1; ++round) {
      for (int pr = warp; pr < npairs; pr += NW) {
        const int c0 = pc0[round][pr], c1 = pc1[round][pr];
        JT* x = X + c0 * KP;
        JT* y = X + c1 * KP;
        const int i0 = lane, i1 = lane + 32;
        const JT x0 = i0 < ke ? x[i0] : JT(0), y0 = i0 < ke ? y[i0] : JT(0);
        const JT x1 = i1 < ke ? x[i1] : JT(0), y1 = i1 < ke ? y[i1] : JT(0);
        JT al = x0 * x0 + x1 * x1, be = y0 * y0 + y1 * y1, ga = x0 * y0 + x1 * y1;
        al = warp_sum_t(al);
        be = warp_sum_t(be);
        ga = warp_sum_t(ga);
        if (ga != JT(0) && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const JT zeta = fdiv_t<JT>(be - al, JT(2) * ga);
          const JT t = fdiv_t<JT>(zeta >= JT(0) ? JT(1) : JT(-1), fabs(zeta) + sqrt(JT(1) + zeta * zeta));
          const JT c = rsqrt_t<JT>(JT(1) + t * t);
          const JT s = c * t;
          JT* zx = Z + c0 * KP;
          JT* zy = Z + c1 * KP;
          if (i0 < ke) {
            x[i0] = c * x0 - s * y0;
            y[i0] = s * x0 + c * y0;
            const JT a = zx[i0], b = zy[i0];
            zx[i0] = c * a - s * b;
            zy[i0] = s * a + c * b;
          }
          if (i1 < ke) {
            x[i1] = c * x1 - s * y1;
            y[i1] = s * x1 + c * y1;
            const JT a = zx[i1], b = zy[i1];
            zx[i1] = c * a - s * b;
            zy[i1] = s * a + c * b;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  __syncthreads();
}

// X <- X P in place (ke x ke, column c at X[c * KP + i]): row i of the
// result depends only on row i of X, so a warp computes a row into
// registers and writes it back.
__device__ void rowwise_product(double* X, const double* P, int ke) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  for (int i = warp; i < ke; i += NW) {
    double a0 = 0.0, a1 = 0.0;
    const int j0 = lane, j1 = lane + 32;
    for (int l = 0; l < ke; ++l) {
      const double x = X[l * KP + i];
      if (j0 < ke) a0 += x * P[j0 * KP + l];
      if (j1 < ke) a1 += x * P[j1 * KP + l];
    }
    __syncwarp();
    if (j0 < ke) X[j0 * KP + i] = a0;
    if (j1 < ke) X[j1 * KP + i] = a1;
  }
  __syncthreads();
}

constexpr int kMixedJacobiMin = 12;  // below, plain float64 sweeps are cheap

// One float32 pass of the mixed Jacobi on a float64 core (see the caller).
__device__ void mixed_rebase_pass(CoreSmem<double>& S, int ke, const unsigned char (*pc0)[KMAX / 2],
                                  const unsigned char (*pc1)[KMAX / 2]) {
  const int tid = threadIdx.x, NT = blockDim.x;
  float* M32 = reinterpret_cast<float*>(S.scrA);
  float* Z32 = M32 + KMAX * KP;
  // scale by a power of two so the largest entry is O(1) in float32
  if (tid == 0) S.amax = 0.0;
  __syncthreads();
  double am = 0.0;
  for (int idx = tid; idx < ke * ke; idx += NT) {
    const int c = idx / ke, i = idx % ke;
    am = fmax(am, fabs(S.Mx[c * KP + i]));
  }
  am = warp_max(am);
  if ((tid & 31) == 0) atomic_max_pos(&S.amax, am);
  __syncthreads();
  const double sc = S.amax > 0.0 ? ldexp(1.0, -ilogb(S.amax)) : 1.0;
  for (int idx = tid; idx < ke * ke; idx += NT) {
    const int c = idx / ke, i = idx % ke;
    M32[c * KP + i] = (float)(S.Mx[c * KP + i] * sc);
    Z32[c * KP + i] = c == i ? 1.f : 0.f;
  }
  __syncthreads();
  const float tol32 = (float)((ke < 4 ? 8 : 2 * ke) * (double)FLT_EPSILON);
  jacobi_sweeps<float>(M32, Z32, ke, tol32, 40, pc0, pc1, &S.flag);
  // Z (float64, in scrB) from the float32 rotations, then two Newton-Schulz
  // steps with the product temporary in scrA (the float32 copies are done).
  double* Zp = S.scrB;
  double* T = S.scrA;
  for (int idx = tid; idx < ke * ke; idx += NT) {
    const int c = idx / ke, i = idx % ke;
    Zp[c * KP + i] = (double)Z32[c * KP + i];
  }
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    // T = (3 I - Z^T Z) / 2, symmetric
    for (int idx = tid; idx < ke * ke; idx += NT) {
      const int a = idx / ke, b = idx % ke;
      if (b > a) continue;
      double g = 0.0;
      for (int i = 0; i < ke; ++i) g += Zp[a * KP + i] * Zp[b * KP + i];
      const double t = (a == b ? 1.5 : 0.0) - 0.5 * g;
      T[a * KP + b] = t;
      T[b * KP + a] = t;
    }
    __syncthreads();
    rowwise_product(Zp, T, ke);
  }
  rowwise_product(S.Mx, Zp, ke);
  rowwise_product(S.Zm, Zp, ke);
}

template <typename T, typename JT>
__device__ __forceinline__ void core_body(const CoreArgs<T>& A);

template <typename T, typename JT>
__global__ void __launch_bounds__(256, 1) core_kernel(CoreArgs<T> A) {
  core_body<T, JT>(A);
}

// One rounding core per CTA for the problems of a batched solve: the skeleton
// of problem blockIdx.x (Gram matrices, weights and k from its cross).
template <typename T, typename JT>
__global__ void __launch_bounds__(256, 1) batch_core_kernel(const BatchProb* __restrict__ P, double eps) {
  const BatchProb& B = P[blockIdx.x];
  CoreArgs<T> A;
  A.GC = B.GC;
  A.GR = B.GR;
  A.ldg = B.kcap;
  A.d = B.d;
  A.k_dev = &B.st->k;
  A.k_host = 0;
  A.eps = eps;
  A.rmax_out = B.ncap;
  A.Tc = static_cast<T*>(B.Tc);
  A.Tr = static_cast<T*>(B.Tr);
  A.s_out = B.so;
  A.st = B.st;
  core_body<T, JT>(A);
}

template <typename T, typename JT>
__device__ __forceinline__ void core_body(const CoreArgs<T>& A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CoreSmem<JT>& S = *reinterpret_cast<CoreSmem<JT>*>(smem_raw);
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
  const int k = A.k_dev ? *A.k_dev : A.k_host;
  if (k <= 0) {
    if (tid == 0) { A.st->rank = 0; A.st->cut = 0; A.st->sigma0 = 0.0; }
    return;
  }
  if (A.tri_given) {
    // GC, GR hold upper-triangular QR factors R_L, R_R of factors with
    // orthonormal Q: take Lc = R_L^T, Lr = R_R^T and skip the Cholesky step.
    for (int idx = tid; idx < k * k; idx += NT) {
      const int i = idx / k, j = idx % k;
      S.Lc[i * KP + j] = j <= i ? A.GC[j + (size_t)i * A.ldg] : 0.0;
      S.Lr[i * KP + j] = j <= i ? A.GR[j + (size_t)i * A.ldg] : 0.0;
    }
    for (int i = tid; i < k; i += NT) S.d[i] = A.d ? A.d[i] : 1.0;
    __syncthreads();
  } else {
  // Load Gram matrices (full, symmetric) and weights.
  for (int idx = tid; idx < k * k; idx += NT) {
    const int i = idx % k, j = idx / k;
    S.Lc[i * KP + j] = A.GC[i + (size_t)j * A.ldg];
    S.Lr[i * KP + j] = A.GR[i + (size_t)j * A.ldg];
  }
  for (int i = tid; i < k; i += NT) {
    S.d[i] = A.d[i];
    S.g0c[i] = A.GC[i + (size_t)i * A.ldg];
    S.g0r[i] = A.GR[i + (size_t)i * A.ldg];
  }
  __syncthreads();
  // Cholesky of both Gram matrices (lower, row-major Lx[i*KP+j], i >= j).
  // A pivot that has lost all but 1e-13 of its original size is lifted to
  // that floor, so an (almost) dependent column gives a tiny singular value
  // that the truncation drops, instead of a breakdown.
  for (int j = 0; j < k; ++j) {
    if (tid < 2) {
      double* L = tid == 0 ? S.Lc : S.Lr;
      const double g0 = tid == 0 ? S.g0c[j] : S.g0r[j];
      double djj = L[j * KP + j];
      const double floor_ = 1e-13 * g0 > DBL_MIN ? 1e-13 * g0 : DBL_MIN;
      if (!(djj > floor_)) djj = floor_;
      const double ljj = sqrt(djj);
      L[j * KP + j] = ljj;
      (tid == 0 ? S.invc : S.invr)[j] = 1.0 / ljj;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < 2 * k; i += NT) {
      if (i < k) S.Lc[i * KP + j] *= S.invc[j];
      else if (i - k > j) S.Lr[(i - k) * KP + j] *= S.invr[j];
    }
    __syncthreads();
    const int rem = k - j - 1;
    for (int idx = tid; idx < 2 * rem * rem; idx += NT) {
      const int side = idx / (rem * rem), w = idx % (rem * rem);
      const int i = j + 1 + w / rem, jj = j + 1 + w % rem;
      if (jj > i) continue;
      double* L = side == 0 ? S.Lc : S.Lr;
      L[i * KP + jj] -= L[i * KP + j] * L[jj * KP + j];
    }
    __syncthreads();
  }
  // Zero the strict upper triangles.
  for (int idx = tid; idx < k * k; idx += NT) {
    const int i = idx / k, j = idx % k;
    if (j > i) { S.Lc[i * KP + j] = 0.0; S.Lr[i * KP + j] = 0.0; }
  }
  __syncthreads();
  }
  // Scale M by a power of two (exact) so that its entries are at most about
  // 1 (|M_pq| <= ||Lc||_F max|d| ||Lr||_F): the iteration in the working
  // precision then never meets values near the ends of its range.
  {
    double a = 0.0, b = 0.0, dm = 0.0;
    for (int idx = tid; idx < k * k; idx += NT) {
      const int i = idx / k, j = idx % k;
      a += S.Lc[i * KP + j] * S.Lc[i * KP + j];
      b += S.Lr[i * KP + j] * S.Lr[i * KP + j];
    }
    for (int i = tid; i < k; i += NT) dm = fmax(dm, fabs(S.d[i]));
    a = warp_sum_t(a);
    b = warp_sum_t(b);
    dm = warp_max(dm);
    if (lane == 0) { S.red[0][warp] = a; S.red[1][warp] = b; S.red[2][warp] = dm; }
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, dm = 0.0;
    for (int w = 0; w < NW; ++w) { a += S.red[0][w]; b += S.red[1][w]; dm = fmax(dm, S.red[2][w]); }
    const double bound = sqrt(a) * sqrt(b) * dm;
    S.scale = (bound > 0.0 && isfinite(bound)) ? ldexp(1.0, -ilogb(bound)) : 1.0;
  }
  __syncthreads();
  const double msc = S.scale;
  // Core M = Lc^T diag(d) Lr : M[p][q] = sum_{i >= max(p,q)} Lc[i][p] d_i Lr[i][q].
  const int ke = k + (k & 1);  // even number of columns for the pairing
  for (int idx = tid; idx < ke * ke; idx += NT) {
    const int p = idx % ke, qq = idx / ke;   // row p, column qq
    double acc = 0.0;
    if (p < k && qq < k) {
      const int i0 = p > qq ? p : qq;
      for (int i = i0; i < k; ++i) acc += S.Lc[i * KP + p] * S.d[i] * S.Lr[i * KP + qq];
    }
    S.Mx[qq * KP + p] = (JT)(acc * msc);
    S.Zm[qq * KP + p] = (JT)(p == qq ? 1.0 : 0.0);
  }
  __syncthreads();
  // Round-robin (circle) pair schedule: in round t, position p meets
  // position ke-1-p; position 0 holds column 0, the others rotate.
  const int npairs = ke / 2;
  __shared__ unsigned char pair_c0[KMAX][KMAX / 2], pair_c1[KMAX][KMAX / 2];
  for (int idx = tid; idx < (ke - 1) * npairs; idx += NT) {
    const int round = idx / npairs, pr = idx % npairs;
    const int pos1 = ke - 1 - pr;
    pair_c0[round][pr] = (unsigned char)(pr == 0 ? 0 : 1 + (pr - 1 + round) % (ke - 1));
    pair_c1[round][pr] = (unsigned char)(1 + (pos1 - 1 + round) % (ke - 1));
  }
  __syncthreads();
  if constexpr (sizeof(JT) == 8) {
    // float64 core: GB300 runs float64 at a small fraction of its float32
    // rate, so most of the iteration runs in float32 on a scaled copy, and
    // float64 only re-bases and polishes:
    //   pass (x2): Z32 = Jacobi_f32(M / 2^e);  Z = NS(NS(Z32))  (Newton-Schulz,
    //              Z <- Z (3 I - Z^T Z) / 2, orthogonal to float64 accuracy);
    //              M <- M Z, Zm <- Zm Z   (float64)
    // The first pass resolves the singular values above ~1e-7 of the largest;
    // after re-basing the small ones sit in columns of their own size, which
    // the second float32 pass resolves in turn; float64 sweeps then finish.
    if (k >= kMixedJacobiMin) {
      for (int pass = 0; pass < 2; ++pass) mixed_rebase_pass(S, ke, pair_c0, pair_c1);
    }
  }
  const JT tol = (JT)((k < 4 ? 8 : 2 * k) * ((sizeof(JT) == 8) ? DBL_EPSILON : (double)FLT_EPSILON));
  jacobi_sweeps<JT>(S.Mx, S.Zm, ke, tol, 40, pair_c0, pair_c1, &S.flag);
  // Singular values (column norms) and their descending order.
  for (int qq = warp; qq < k; qq += NW) {
    double acc = 0.0;
    for (int i = lane; i < k; i += 32) acc += (double)S.Mx[qq * KP + i] * (double)S.Mx[qq * KP + i];
    acc = warp_sum_t(acc);
    // A non-finite value (overflow or 0/0 upstream) is ranked last as -1, so
    // the ordering below stays a permutation; the solve is then failed.
    if (lane == 0) S.sig[qq] = isfinite(acc) ? sqrt(acc) / msc : -1.0;
  }
  __syncthreads();
  for (int qq = tid; qq < k; qq += NT) {
    int rank = 0;
    for (int p = 0; p < k; ++p)
      if (S.sig[p] > S.sig[qq] || (S.sig[p] == S.sig[qq] && p < qq)) ++rank;
    S.perm[rank] = qq;
  }
  __syncthreads();
  if (tid == 0) {
    double total = 0.0;
    for (int p = 0; p < k; ++p) total += S.sig[p] * S.sig[p];
    int K;
    if (S.sig[S.perm[0]] == 0.0 || S.sig[S.perm[k - 1]] < 0.0) {
      K = 0;
      if (S.sig[S.perm[k - 1]] < 0.0) A.st->status = LR_ENONFINITE;
    } else {
      const double lim = fmax(A.eps * sqrt(total), A.eps_abs);
      double tail2 = 0.0;
      K = k;
      for (int p = k - 1; p >= 1; --p) {
        const double sp = S.sig[S.perm[p]];
        const double t2 = tail2 + sp * sp;
        if (sqrt(t2) > lim) break;
        tail2 = t2;
        K = p;
      }
    }
    const int cut = K > A.rmax_out;
    if (cut) K = A.rmax_out;
    S.K = K;
    A.st->rank = K;
    A.st->cut = cut;
    A.st->sigma0 = K > 0 ? S.sig[S.perm[0]] : 0.0;
  }
  __syncthreads();
  const int K = S.K;
  for (int p = tid; p < K; p += NT) A.s_out[p] = S.sig[S.perm[p]];
  // Tc = Lc^-T W_K (W column p = M column perm[p] / sig), Tr = Lr^-T Z_K.
  for (int job = tid; job < 2 * K; job += NT) {
    const int side = job / K, p = job % K;
    const int src = S.perm[p];
    const double* L = side == 0 ? S.Lc : S.Lr;
    const double* inv_diag = side == 0 ? S.invc : S.invr;
    T* out = side == 0 ? A.Tc : A.Tr;
    const double inv = side == 0 ? (S.sig[src] > 0.0 ? 1.0 / (S.sig[src] * msc) : 0.0) : 1.0;
    const JT* col = side == 0 ? S.Mx + src * KP : S.Zm + src * KP;
    if (A.tri_given) {  // the factors are already orthonormal: T = W_K, Z_K
      for (int i = 0; i < k; ++i) out[i + (size_t)p * KMAX] = (T)((double)col[i] * inv);
      continue;
    }
    // back substitution with L^T (upper triangular): x_i = (w_i - sum_{j>i} L[j][i] x_j) / L[i][i]
    double xs[KMAX];
    for (int i = k - 1; i >= 0; --i) {
      double acc = (double)col[i] * inv;
      for (int j = i + 1; j < k; ++j) acc -= L[j * KP + i] * xs[j];
      xs[i] = acc * inv_diag[i];
    }
    for (int i = 0; i < k; ++i) out[i + (size_t)p * KMAX] = (T)xs[i];
  }
}

template <typename T>
cudaError_t launch_core(const CoreArgs<T>& a, bool jacobi_fp32, cudaStream_t st) {
  if (jacobi_fp32) {
    auto kern = core_kernel<T, float>;
    const size_t sm = sizeof(CoreSmem<float>);
    static cudaError_t set = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (set != cudaSuccess) return set;
    kern<<<1, 256, sm, st>>>(a);
  } else {
    auto kern = core_kernel<T, double>;
    const size_t sm = sizeof(CoreSmem<double>);
    static cudaError_t set = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (set != cudaSuccess) return set;
    kern<<<1, 256, sm, st>>>(a);
  }
  return cudaGetLastError();
}
template cudaError_t launch_core<double>(const CoreArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_core<float>(const CoreArgs<float>&, bool, cudaStream_t);

template <typename T>
cudaError_t launch_batch_core(const BatchProb* probs, int n, double eps, bool jacobi_fp32, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (jacobi_fp32) {
    auto kern = batch_core_kernel<T, float>;
    const size_t sm = sizeof(CoreSmem<float>);
    static cudaError_t set = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (set != cudaSuccess) return set;
    kern<<<n, 256, sm, st>>>(probs, eps);
  } else {
    auto kern = batch_core_kernel<T, double>;
    const size_t sm = sizeof(CoreSmem<double>);
    static cudaError_t set = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (set != cudaSuccess) return set;
    kern<<<n, 256, sm, st>>>(probs, eps);
  }
  return cudaGetLastError();
}
template cudaError_t launch_batch_core<double>(const BatchProb*, int, double, bool, cudaStream_t);
template cudaError_t launch_batch_core<float>(const BatchProb*, int, double, bool, cudaStream_t);

// ---------------------------------------------------------------------------
// Gram matrix G = X^T X of a tall float64 matrix: per-block partial sums in a
// fixed order, then a deterministic sum over blocks.
// ---------------------------------------------------------------------------
constexpr int kGramRows = 64;

__global__ void __launch_bounds__(256) gram_partial_kernel(const double* __restrict__ X, int rows, int ld,
                                                           int k, double* __restrict__ partial) {
  __shared__ double tile[kGramRows * KMAX];
  const int r0 = blockIdx.x * kGramRows;
  const int nr = min(kGramRows, rows - r0);
  for (int idx = threadIdx.x; idx < kGramRows * k; idx += blockDim.x) {
    const int i = idx % kGramRows, l = idx / kGramRows;
    tile[l * kGramRows + i] = i < nr ? X[(size_t)l * ld + r0 + i] : 0.0;
  }
  __syncthreads();
  double* out = partial + (size_t)blockIdx.x * KMAX * KMAX;
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int p = idx % k, q = idx / k;
    if (p > q) continue;
    double acc = 0.0;
    for (int i = 0; i < nr; ++i) acc += tile[p * kGramRows + i] * tile[q * kGramRows + i];
    out[p + q * KMAX] = acc;
  }
}

__global__ void gram_sum_kernel(const double* __restrict__ partial, int nblk, int k, double* __restrict__ G,
                                int ldg) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < k * k; idx += gridDim.x * blockDim.x) {
    const int p = idx % k, q = idx / k;
    if (p > q) continue;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += partial[(size_t)b * KMAX * KMAX + p + q * KMAX];
    G[p + (size_t)q * ldg] = acc;
    G[q + (size_t)p * ldg] = acc;
  }
}

cudaError_t launch_gram(const double* X, int rows, int ld, int k, double* G, int ldg, double* partial,
                        int num_sms, cudaStream_t st) {
  (void)num_sms;
  const int nblk = (rows + kGramRows - 1) / kGramRows;
  gram_partial_kernel<<<nblk, 256, 0, st>>>(X, rows, ld, k, partial);
  gram_sum_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(partial, nblk, k, G, ldg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rotation out[:, q] = sum_{l<k} in[:, l] Tm[l, q], q < rank (device values).
// ---------------------------------------------------------------------------
template <typename TI, typename TO, typename TM>
__global__ void __launch_bounds__(256) rotate_kernel(const TI* __restrict__ in, int ld_in, int rows,
                                                     const int* k_dev, int k_host, const TM* __restrict__ Tm,
                                                     const int* rank_dev, TO* __restrict__ out, int ld_out) {
  __shared__ TM tm[KMAX * KMAX];
  const int k = k_dev ? *k_dev : k_host;
  const int R = *rank_dev;
  for (int idx = threadIdx.x; idx < k * R; idx += blockDim.x) {
    const int l = idx % k, qq = idx / k;
    tm[l + qq * KMAX] = Tm[l + (size_t)qq * KMAX];
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  for (int q0 = 0; q0 < R; q0 += 8) {
    TM acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = TM(0);
    for (int l = 0; l < k; ++l) {
      const TM x = (TM)in[row + (size_t)l * ld_in];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] += x * tm[l + (q0 + c) * KMAX];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (q0 + c < R) out[row + (size_t)(q0 + c) * ld_out] = (TO)acc[c];
  }
}

template <typename TI, typename TO>
cudaError_t launch_rotate(const TI* in, int ld_in, int rows, const int* k_dev, int k_host, const void* Tm,
                          bool tm_f32, const int* rank_dev, TO* out, int ld_out, cudaStream_t st) {
  const int grid = (rows + 255) / 256;
  if (tm_f32)
    rotate_kernel<TI, TO, float><<<grid, 256, 0, st>>>(in, ld_in, rows, k_dev, k_host,
                                                       static_cast<const float*>(Tm), rank_dev, out, ld_out);
  else
    rotate_kernel<TI, TO, double><<<grid, 256, 0, st>>>(in, ld_in, rows, k_dev, k_host,
                                                        static_cast<const double*>(Tm), rank_dev, out, ld_out);
  return cudaGetLastError();
}
template cudaError_t launch_rotate<double, double>(const double*, int, int, const int*, int, const void*, bool,
                                                   const int*, double*, int, cudaStream_t);
template cudaError_t launch_rotate<float, float>(const float*, int, int, const int*, int, const void*, bool,
                                                 const int*, float*, int, cudaStream_t);

}  // namespace lrp
