// Internal interfaces between the translation units of liblrpoisson.so.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "lr_common.cuh"

namespace lrp {

// ---------------------------------------------------------------------------
// Sine-transform plan: tables for the Bluestein evaluation of the DST-I of
// order m (Section 4.1) with a power-of-two FFT of length M >= 2m - 1.
//   chirp[t]  = exp(i pi (t+1)^2 / (2N)), N = m + 1, t < m
//   tw[q]     = exp(-2 pi i q / M), q < M
//   bhat      = FFT_M of the chirp kernel conj(w_|d|), |d| < m, scaled by
//               sqrt(2/N)/M; natural order if M <= kSmallM, else stored as
//               [k2][k1] for the four-step split M = M1 * M2.
// Symbol tables: Lambda[i,j] = a_i b_j + b_i a_j (both operator kinds).
// ---------------------------------------------------------------------------
constexpr int kSmallM = 4096;      // one CTA holds a whole length-M sequence
// One-pass batched transform (float32): FFT length H <= 2^kFusedLogH32 held
// whole in one CTA's shared memory; longer M split into M / H residues.
constexpr int kFusedLogH32 = 14;
constexpr int kTileElems = 4096;   // complex elements per CTA tile
constexpr int kFftThreads = 256;   // 16 elements per thread

struct TablesT {
  void* chirp = nullptr;  // cpx<T>[m]
  void* tw = nullptr;     // cpx<T>[M]
  void* bhat = nullptr;   // cpx<T>[M]
  void* bhat_cl = nullptr;  // cpx<T>[M], cluster order [k1][k2] (cluster path only)
  void* bhat_rs = nullptr;  // cpx<T>[M], float32 only, order of the one-pass transform:
                            // residue t of R = M / H (H = min(M, 2^kFusedLogH32)), then
                            // the digit-reversed position p of its length-H FFT:
                            // [t][p] = b[R inplace_freq(p) + t]
  void* a = nullptr;      // T[m] per operator kind (index by op)
  void* b = nullptr;
};

struct Plan {
  int m = 0;
  int logM = 0, logM1 = 0, logM2 = 0;
  TablesT t64, t32;                       // float64 and float32 copies
  double* sym_a64[2] = {nullptr, nullptr};  // per operator kind
  double* sym_b64[2] = {nullptr, nullptr};
  float* sym_a32[2] = {nullptr, nullptr};
  float* sym_b32[2] = {nullptr, nullptr};
  int log_tile[2] = {0, 0};                 // tuned four-step tile (0: heuristic), [fp64, fp32]
  int logN2cl = 0;                          // cluster-path chunk (0: no cluster path)
  int use_cluster[2] = {0, 0};              // transform variant: 1 = cluster path, [fp64, fp32]
  std::vector<void*> allocations;
  ~Plan();
};

std::string build_plan(int m, Plan& p);   // returns "" on success

// A set of columns to transform: segment 0 has ncol0 columns, segment 1
// ncol1 columns.  If dyn_count is non-null the number of live columns of each
// segment is *dyn_count (read on the device) and ncol0/ncol1 are capacities.
struct ColumnSet {
  const void* in[2] = {nullptr, nullptr};
  void* out[2] = {nullptr, nullptr};
  int ld_in[2] = {0, 0};
  int ld_out[2] = {0, 0};
  int ncol[2] = {0, 0};
  const int* dyn_count = nullptr;
  // IoType::ROT input: column q of segment s is sum_{l<k} in[s][:, l] tm[s][l + q*KMAX]
  // (working precision, k read from *k_dev on the device).
  const void* tm[2] = {nullptr, nullptr};
  const int* k_dev = nullptr;
  // IoType::DIV input: element t of column q is in[s][t + q ld] / (a_t b_q + b_t a_q)
  // (working-precision symbol tables a, b: the division by Lambda of Eq. flr:diag)
  const void* sym_a = nullptr;
  const void* sym_b = nullptr;
};

// Input/output kinds: caller float64 buffers, working-precision buffers, or
// (input only) working-precision columns rotated on the fly, or divided by
// the symbol on the fly.
enum class IoType { F64, WORK, ROT, DIV };

// Launch the DST-I of every column of cs (forward and inverse are the same
// orthonormal, symmetric S).  work: complex scratch of M * (ncol0 + ncol1)
// elements of the working precision.  Returns a CUDA error code.
template <typename T>
cudaError_t launch_dst(const Plan& p, const ColumnSet& cs, IoType in_t, IoType out_t,
                       void* work, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------------------
// Cross approximation in frequency space (Section 4.2).
// ---------------------------------------------------------------------------
template <typename T>
struct CrossArgs {
  int m, r, kcap, ld;
  const T* Uh;
  const T* Vh;
  T* C;            // m x kcap, column l: residual column / delta_l
  T* R;            // m x kcap, column l: residual row / delta_l
  const T* a;      // symbol
  const T* b;
  double* d;       // kcap pivot values
  int* I;
  int* J;
  double* GC;      // kcap x kcap Gram matrices (column-major, ld kcap)
  double* GR;
  SolveState* st;
  double tol;
  int probes;
  unsigned long long seed;
  int max_probe_rounds;
  int max_zero_rows;
};

template <typename T>
cudaError_t launch_cross(const CrossArgs<T>& a, int cluster_size, cudaStream_t st, int* used_cluster);

// ---------------------------------------------------------------------------
// Rounding core (Section 3): Cholesky of the Gram matrices, SVD of the k x k
// core, truncation, coefficient matrices Tc, Tr (k x R, ld KMAX).
// ---------------------------------------------------------------------------
template <typename T>
struct CoreArgs {
  const double* GC;
  const double* GR;
  int ldg;          // leading dimension of GC/GR
  const double* d;  // weights (k)
  const int* k_dev; // k on the device (nullptr: use k_host)
  int k_host;
  double eps;
  int rmax_out;
  T* Tc;            // KMAX x KMAX
  T* Tr;
  double* s_out;    // R singular values
  SolveState* st;
  double eps_abs = 0.0; // if > 0: also drop singular values while the dropped
                        // tail stays within eps_abs (absolute)
  int tri_given = 0; // 1: GC, GR are upper-triangular QR factors (column-major,
                     // ldg), d may be null (ones); T = W_K, Z_K directly
};
template <typename T>
cudaError_t launch_core(const CoreArgs<T>& a, bool jacobi_fp32, cudaStream_t st);

// Gram matrices of two tall factors (float64): G = X^T X.
cudaError_t launch_gram(const double* X, int rows, int ld, int k, double* G, int ldg,
                        double* partial, int num_sms, cudaStream_t st);

// Rotation: out[:, q] = sum_l in[:, l] * Tm[l, q] for q < rank (rank on the device).
template <typename TI, typename TO>
cudaError_t launch_rotate(const TI* in, int ld_in, int rows, const int* k_dev, int k_host,
                          const void* Tm, bool tm_f32, const int* rank_dev, TO* out, int ld_out,
                          cudaStream_t st);

// Stokes (Section 2): bidiagonal maps of factor columns, cross Gram matrices,
// column sums against the pressure's kernel modes.
enum : int { OP_G = 0, OP_H = 1, OP_GT = 2, OP_HT = 3 };
cudaError_t launch_gh(int op, int n, const double* in, int ldi, int r, const double* w, double scale,
                      double* out, int ldo, cudaStream_t st);
cudaError_t launch_cross_gram(const double* X, int ldx, const double* Y, int ldy, int rows, int kx, int ky,
                              double* C, double* partial, cudaStream_t st);
cudaError_t launch_colsums(const double* X, int ld, int rows, int r, double* out, cudaStream_t st);
cudaError_t launch_kernel_modes(int rows, double* e, int ld, cudaStream_t st);
cudaError_t launch_scale_copy(int n, const double* src, double coef, double* dst, cudaStream_t st);

// out[j + i ldo] = in[i + j ldi] for an m x n working-precision matrix.
template <typename T>
cudaError_t launch_transpose(const T* in, int ldi, int m, int n, T* out, int ldo, cudaStream_t st);

// Iterative refinement helpers (float64): the residual F - A X as factors
// [UF, -c P U s, -c Q U s], [VF, Q V, P V] (r + 2R columns, leading dim ldo).
cudaError_t launch_residual_factors(int m, int r, int R, const double* UF, const double* VF, int ldf,
                                    const double* U, const double* s, const double* V, int ldx, int op,
                                    double* L, double* Rt, int ldo, cudaStream_t st);
// One shifted/plain Cholesky QR step on two factors (see refine.cu).
struct CholQrArgs {
  const double* G[2];  // q x q Gram matrices (ld q)
  double* T[2];        // KMAX x KMAX: X T has orthonormal columns
  double* Racc[2];     // KMAX x KMAX: accumulated upper-triangular R
  int* qout;           // [2], set to q (rotation column count)
  int q;
  int first;           // 1: Racc = this step's R
  double shift;        // added to the equilibrated Gram diagonal
  double floor_rel;    // Cholesky pivots at or below are dropped columns
};
cudaError_t launch_cholqr_step(const CholQrArgs& a, cudaStream_t st);
cudaError_t launch_fold_weights(int m, int kmax, const int* K, double* U, int ld, const double* s, bool unit,
                                cudaStream_t st);
cudaError_t launch_scale_weights(int n, double* w, const double* s, cudaStream_t st);
cudaError_t launch_expsum_cols(int m, int r, int nterms, const double* Uh, const double* Vh, int ldh,
                               const double* mu, const double* t, const double* w, double* L, double* R, int ldo,
                               int off, cudaStream_t st);

// ---------------------------------------------------------------------------
// Phase-batched solves (batch.cu): every step of the Section 4.2 solve for all
// problems of a batch in one launch per step.  Each problem is described on
// the device by a BatchProb; the working-precision buffers are T* of the
// launch's precision.
// ---------------------------------------------------------------------------
struct BatchProb {
  int m, r, kcap, ldw;       // order, RHS rank, cross step cap, ld of working buffers
  int ncap;                  // output columns (min(kcap, sol->rmax))
  int logM, logM1, logM2;    // transform length M = 2^logM = M1 * M2
  int ld_in, ld_out;
  const double* U;           // right-hand side factors (caller, float64)
  const double* V;
  double* Uo;                // solution factors and singular values (caller)
  double* Vo;
  double* so;
  void* Uh;                  // m x r transformed factors
  void* Vh;
  void* C;                   // m x kcap skeleton factors
  void* R;
  void* Tc;                  // KMAX x KMAX rotations of the rounding core
  void* Tr;
  void* W;                   // m x 2 ncap rotated skeleton (inverse transform input)
  void* work;                // four-step scratch, M complex per column
  double* GC;                // kcap x kcap Gram matrices
  double* GR;
  double* d;                 // pivot values
  int* I;
  int* J;
  SolveState* st;
  const void* chirp;         // plan tables of the working precision
  const void* tw;
  const void* bhat;
  const void* bres;          // kernel spectrum in residue order (one-pass transform)
  const void* sa;            // symbol of the operator kind
  const void* sb;
};

// Item lists of one batched launch: the problems taking part (list[q]) and
// the first item of each (start[q], start[n] = total items).
struct BatchItems {
  const int* list = nullptr;
  const int* start = nullptr;
  int n = 0;
  int items = 0;     // items, or (live lists) the capacity the grid is sized for
  int live = 0;      // 1: start[] is written on the device by launch_batch_live_items
                     // and counts only the live (rank < R) columns, start[n] = items
  int slog = 0;      // largest log2 sub-length of the launch's FFT stages (log2 L - 2)
  int fused_logh = 0;  // column list of the one-pass transform (FFT length cap
                       // 2^fused_logh, one item per 2^(fused_logh - min(logM,
                       // fused_logh)) columns); 0: four-step passes
};

// Item tables of the inverse transforms over live columns only: for each of
// the lists (small, column pass, row pass) start[q] = sum over earlier
// problems of their live items (2 R columns, R the kept rank).
cudaError_t launch_batch_live_items(const BatchProb* probs, const BatchItems& small, const BatchItems& col,
                                    const BatchItems& row, cudaStream_t st);

// Batched sine transforms of all problems' columns (dir 0: U, V -> Uh, Vh;
// dir 1: the rotated skeleton W -> the caller's solution factors, live
// columns < rank).  small: problems with M <= 4096 (items of 4096 / M
// columns); col, row: four-step problems (col: column-pass items, row:
// row-pass items, same list).  tw4096: twiddles exp(-2 pi i q / 4096).
template <typename T>
cudaError_t launch_batch_dst(const BatchProb* probs, int dir, const BatchItems& small, const BatchItems& col,
                             const BatchItems& row, const void* tw4096, int num_sms, cudaStream_t st);

// Batched rotation W = [C Tc, R Tr] (rows < m, columns < rank) of every
// problem; items: row blocks of 256.
template <typename T>
cudaError_t launch_batch_rotate(const BatchProb* probs, const BatchItems& rows, int num_sms, cudaStream_t st);

struct BatchCrossParams {
  double tol;
  int probes;
  unsigned long long seed;
  int max_probe_rounds;
  int max_zero_rows;
};

// Batched cross: problems list[0..n) (LPT order), each on a cluster of cs
// CTAs (1, 2, 4, 8 or 16) with rows_per_cta >= ceil(m / cs) indices per CTA.
template <typename T>
cudaError_t launch_batch_cross(const BatchProb* probs, const int* list, int n, int cs, int rows_per_cta,
                               const BatchCrossParams& cp, cudaStream_t st);
// Largest indices per CTA the batched cross supports in this precision.
int batch_cross_max_rows(bool f32);

// Batched rounding cores, one CTA per problem (core.cu).
template <typename T>
cudaError_t launch_batch_core(const BatchProb* probs, int n, double eps, bool jacobi_fp32, cudaStream_t st);

// ---- 3D Tucker solve (tucker.cu) -------------------------------------------
constexpr int T3P = KMAX;  // largest basis size per mode; stride of core-sized tensors

// Device state of one Tucker cross.
struct T3State {
  int pos[3];        // search position (i, j, k)
  int p[3];          // basis sizes
  int add[3];        // the step's fibre of this mode enters the basis
  int negl;          // the step's pivot is negligible
  int done, converged;
  int small;         // consecutive steps that passed the step test (2: probe)
  int probe_rounds;
  int steps;
  int status;        // lr_status of a failure (LR_ENONFINITE)
  double fval[3];    // value at the argmax of the last fibre of each mode
  double fnrm2[3];   // square norm of that fibre
  double rho, rho0;  // pivot of the step, size of the first pivot (-1: none yet)
  double upd, nrmC, est;
};

struct T3Dev {
  int n[3], r[3], ldu[3], ldq[3];
  const double* Uh[3];    // transformed factors of the right-hand side, n_k x r_k (ld ldu)
  const double* G;        // its core, C order: G[(a r1 + b) r2 + c]
  const double* mu[3];    // 1D symbols (n_k)
  double* Q[3];           // bases n_k x T3P (ld ldq)
  double* Minv[3];        // Q_k(I_k, :)^-1, T3P x T3P column-major
  int* I[3];              // interpolation indices
  unsigned char* inI[3];  // membership of I_k (n_k bytes)
  double* e[3];           // residual fibres of the step
  double* v[3];           // their working copies (orthogonalisation, DEIM residual)
  double* h[3];           // Gram-Schmidt coefficients (T3P)
  double* y[3];           // M_k Q_k(I_k, p_k) (T3P)
  double* C;              // core, C[x0 + T3P (x1 + T3P x2)]
  T3State* st;
};

// out = in x_mode A (see t3_modeprod_kernel).
struct T3ModeProd {
  const double* in;
  int is[3];
  double* out;
  int os[3];
  int od[3];
  int mode, K;
  const double* A;
  const int* rowmap;
  int ars, acs;
  int divlam;
  int skip_negl = 0;
};

struct T3ProbeCounts {
  int nrand[3];
  int ncross[3];
};

cudaError_t launch_t3_search(const T3Dev& d, cudaStream_t st);
cudaError_t launch_t3_probe(const T3Dev& d, int nfib, const int* jobs, double* nrm2, int* amax, cudaStream_t st);
cudaError_t launch_t3_pivot(const T3Dev& d, cudaStream_t st);
cudaError_t launch_t3_basis_update(const T3Dev& d, int nmax, cudaStream_t st);
cudaError_t launch_t3_modeprod(const T3ModeProd& a, const T3Dev& d, cudaStream_t st);
cudaError_t launch_t3_decide(const T3Dev& d, double tol, cudaStream_t st);
cudaError_t launch_t3_probe_reduce(const T3Dev& d, const int* jobs, const double* nrm2, const int* amax,
                                   const T3ProbeCounts& c, double tol, cudaStream_t st);
cudaError_t launch_t3_unfold(const T3Dev& d, int m, int total, double* A, int lda, cudaStream_t st);
cudaError_t launch_t3_widen(const float* in, double* out, int n, cudaStream_t st);

}  // namespace lrp
