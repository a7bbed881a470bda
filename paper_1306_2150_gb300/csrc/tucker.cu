// Kernels of the low-rank 3D Poisson solve in Tucker format (Section 3,
// Eq. flr:tucker; Sections 4.1 and 4.2 in three dimensions): the Tucker
// fibre cross of Xh(i, j, k) = Fh(i, j, k) / (mu_i + mu_j + mu_k) with
// Fh = G x_1 Uh_1 x_2 Uh_2 x_3 Uh_3, and the mode products of its core.
//
// The paper cites a Tucker cross but prints none; the cross built here (its
// steps are listed at t3_* below and in the host driver):
//   * bases Q_k with orthonormal columns, interpolation indices I_k (the DEIM
//     index of each new basis vector, Chaturantabut and Sorensen 2010) and
//     the inverses M_k = Q_k(I_k, :)^-1, updated by bordering;
//   * core C = Xh(I_1, I_2, I_3) x_1 M_1 x_2 M_2 x_3 M_3, so that C x_k Q_k
//     interpolates Xh on I_1 x I_2 x I_3;
//   * a residual fibre R(:, j, k) = Xh(:, j, k) - Q_1 (C x_2 Q_2(j, :) x_3
//     Q_3(k, :)) costs O(p^3 + r^3 + n (p + r)).
// float64 throughout.  Tensors of the core's size are stored with mode 0
// fastest and stride T3P per mode: X[x0 + T3P (x1 + T3P x2)].
#include <algorithm>

#include <cooperative_groups.h>

#include "lr_internal.h"

namespace cg = cooperative_groups;

namespace lrp {

namespace {

constexpr int FT = 256;  // threads of the fibre kernels

__device__ inline void other_modes(int m, int& oa, int& ob) {
  oa = m == 0 ? 1 : 0;
  ob = m == 2 ? 1 : 2;
}

// Block reduction of (sum, argmax |v| with its value, lowest index on ties)
// in a fixed order.
struct RedSmem {
  double s[FT];
  double a[FT];
  double v[FT];
  int i[FT];
};

__device__ void block_reduce(RedSmem& R, double s, double a, double v, int idx) {
  const int t = threadIdx.x;
  R.s[t] = s;
  R.a[t] = a;
  R.v[t] = v;
  R.i[t] = idx;
  __syncthreads();
  for (int o = FT / 2; o > 0; o >>= 1) {
    if (t < o) {
      R.s[t] += R.s[t + o];
      const double a2 = R.a[t + o];
      const int i2 = R.i[t + o];
      if (a2 > R.a[t] || (a2 == R.a[t] && i2 >= 0 && (R.i[t] < 0 || i2 < R.i[t]))) {
        R.a[t] = a2;
        R.v[t] = R.v[t + o];
        R.i[t] = i2;
      }
    }
    __syncthreads();
  }
}

struct FibreSmem {
  double qa[T3P], qb[T3P], ua[T3P], ub[T3P];
  double part[T3P * T3P];
  double cvec[T3P], gvec[T3P];
  RedSmem red;
  int bad;
};

// One residual fibre along mode m at the other two indices (a, b) (a on the
// lower other mode): writes it to e_out / v_out (if non-null) and returns, on
// thread 0, its square norm, the argmax of |value| outside excl and that
// value.
__device__ void t3_fibre(const T3Dev& d, FibreSmem& S, int m, int a, int b, const unsigned char* excl,
                         double* e_out, double* v_out, double* nrm2, int* amax, double* vmax) {
  const int tid = threadIdx.x;
  int oa, ob;
  other_modes(m, oa, ob);
  const int pm = d.st->p[m], pa = d.st->p[oa], pb = d.st->p[ob];
  const int rm = d.r[m], ra = d.r[oa], rb = d.r[ob];
  if (tid == 0) S.bad = 0;
  for (int x = tid; x < T3P; x += FT) {
    S.qa[x] = x < pa ? d.Q[oa][a + (size_t)x * d.ldq[oa]] : 0.0;
    S.qb[x] = x < pb ? d.Q[ob][b + (size_t)x * d.ldq[ob]] : 0.0;
    S.ua[x] = x < ra ? d.Uh[oa][a + (size_t)x * d.ldu[oa]] : 0.0;
    S.ub[x] = x < rb ? d.Uh[ob][b + (size_t)x * d.ldu[ob]] : 0.0;
  }
  __syncthreads();
  // c[xm] = sum_{xa, xb} C[xm, xa, xb] qa[xa] qb[xb]
  const size_t sc[3] = {1, (size_t)T3P, (size_t)T3P * T3P};
  for (int w = tid; w < pm * pa; w += FT) {
    const int xm = w % pm, xa = w / pm;
    const double* c = d.C + xm * sc[m] + xa * sc[oa];
    double acc = 0.0;
    for (int xb = 0; xb < pb; ++xb) acc += c[xb * sc[ob]] * S.qb[xb];
    S.part[xm + T3P * xa] = acc * S.qa[xa];
  }
  __syncthreads();
  for (int xm = tid; xm < pm; xm += FT) {
    double s = 0.0;
    for (int xa = 0; xa < pa; ++xa) s += S.part[xm + T3P * xa];
    S.cvec[xm] = s;
  }
  __syncthreads();
  // g[ym] = sum_{ya, yb} G[ym, ya, yb] ua[ya] ub[yb] (G in C order r0 x r1 x r2)
  const size_t sg[3] = {(size_t)d.r[1] * d.r[2], (size_t)d.r[2], 1};
  for (int w = tid; w < rm * ra; w += FT) {
    const int ym = w % rm, ya = w / rm;
    const double* g = d.G + ym * sg[m] + ya * sg[oa];
    double acc = 0.0;
    for (int yb = 0; yb < rb; ++yb) acc += g[yb * sg[ob]] * S.ub[yb];
    S.part[ym + T3P * ya] = acc * S.ua[ya];
  }
  __syncthreads();
  for (int ym = tid; ym < rm; ym += FT) {
    double s = 0.0;
    for (int ya = 0; ya < ra; ++ya) s += S.part[ym + T3P * ya];
    S.gvec[ym] = s;
  }
  __syncthreads();
  const double lab = d.mu[oa][a] + d.mu[ob][b];
  const int n = d.n[m];
  const double* U = d.Uh[m];
  const double* Qm = d.Q[m];
  const double* mu = d.mu[m];
  double s2 = 0.0, best = -1.0, bestv = 0.0;
  int besti = -1;
  for (int i = tid; i < n; i += FT) {
    double f = 0.0;
    for (int y = 0; y < rm; ++y) f += U[i + (size_t)y * d.ldu[m]] * S.gvec[y];
    double yv = 0.0;
    for (int x = 0; x < pm; ++x) yv += Qm[i + (size_t)x * d.ldq[m]] * S.cvec[x];
    const double val = f / (mu[i] + lab) - yv;
    if (!isfinite(val)) S.bad = 1;
    if (e_out) e_out[i] = val;
    if (v_out) v_out[i] = val;
    s2 += val * val;
    if (!(excl && excl[i])) {
      const double av = fabs(val);
      if (av > best) { best = av; bestv = val; besti = i; }
    }
  }
  block_reduce(S.red, s2, best, bestv, besti);
  if (tid == 0) {
    *nrm2 = S.red.s[0];
    *amax = S.red.i[0] >= 0 ? S.red.i[0] : 0;
    *vmax = S.red.v[0];
    if (S.bad) d.st->status = LR_ENONFINITE;
  }
}

// ---------------------------------------------------------------------------
// The pivot search of one step, on one thread-block cluster of SCS CTAs:
// two rounds of the mode-2, mode-3 and mode-1 fibres (each fibre's argmax
// becoming the position's coordinate in its mode), then the mode-2 and
// mode-3 fibres through the pivot.  Per fibre, the contraction outputs
// c = C x qa x qb and g = G x ua x ub are spread over the cluster's warps and
// gathered through distributed shared memory, the n entries are split in
// contiguous chunks over the CTAs, and the per-CTA (square norm, argmax)
// partials are combined in rank order by every CTA, so all take the same
// decision.  float64 runs at a few FMAs per clock per SM on this part: one
// SM per fibre would make the search the slowest step of the solve.
// ---------------------------------------------------------------------------
constexpr int SCS = 8;          // CTAs in the search cluster
constexpr int SNW = FT / 32;    // warps per CTA

struct SearchSmem {
  double qa[T3P], qb[T3P], ua[T3P], ub[T3P];
  double item[2 * T3P];         // contraction outputs computed here (c, then g)
  double cvec[T3P], gvec[T3P];
  RedSmem red;
  double ps, pa, pv;            // this CTA's partial: square norm, |max|, value
  int pi;                       // and index of the max
  int pos[3];
  int bad;
};

__device__ void cluster_fibre(const T3Dev& d, SearchSmem& S, cg::cluster_group& cl, int m, int a, int b,
                              double* e_out, double* v_out, double* nrm2, int* amax, double* vmax) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = (int)cl.block_rank();
  int oa, ob;
  other_modes(m, oa, ob);
  const int pm = d.st->p[m], pa = d.st->p[oa], pb = d.st->p[ob];
  const int rm = d.r[m], ra = d.r[oa], rb = d.r[ob];
  if (tid == 0) S.bad = 0;
  for (int x = tid; x < T3P; x += FT) {
    S.qa[x] = x < pa ? d.Q[oa][a + (size_t)x * d.ldq[oa]] : 0.0;
    S.qb[x] = x < pb ? d.Q[ob][b + (size_t)x * d.ldq[ob]] : 0.0;
    S.ua[x] = x < ra ? d.Uh[oa][a + (size_t)x * d.ldu[oa]] : 0.0;
    S.ub[x] = x < rb ? d.Uh[ob][b + (size_t)x * d.ldu[ob]] : 0.0;
  }
  __syncthreads();
  // item t < pm: c[t]; pm <= t < pm + rm: g[t - pm]; one warp per item
  const size_t sc[3] = {1, (size_t)T3P, (size_t)T3P * T3P};
  const size_t sg[3] = {(size_t)d.r[1] * d.r[2], (size_t)d.r[2], 1};
  const int items = pm + rm;
  for (int t = rank * SNW + warp; t < items; t += SCS * SNW) {
    double acc = 0.0;
    if (t < pm) {
      const double* c = d.C + t * sc[m];
      for (int w = lane; w < pa * pb; w += 32) {
        const int xa = w % pa, xb = w / pa;
        acc += c[xa * sc[oa] + xb * sc[ob]] * S.qa[xa] * S.qb[xb];
      }
    } else {
      const double* g = d.G + (t - pm) * sg[m];
      for (int w = lane; w < ra * rb; w += 32) {
        const int ya = w % ra, yb = w / ra;
        acc += g[ya * sg[oa] + yb * sg[ob]] * S.ua[ya] * S.ub[yb];
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) S.item[t] = acc;
  }
  cl.sync();
  for (int t = tid; t < items; t += FT) {
    const int owner = (t % (SCS * SNW)) / SNW;
    const double v = *cl.map_shared_rank(&S.item[t], owner);
    if (t < pm) S.cvec[t] = v;
    else S.gvec[t - pm] = v;
  }
  __syncthreads();
  const int n = d.n[m];
  const int chunk = (n + SCS - 1) / SCS;
  const int i0 = rank * chunk, i1 = min(n, i0 + chunk);
  const double lab = d.mu[oa][a] + d.mu[ob][b];
  const double* U = d.Uh[m];
  const double* Qm = d.Q[m];
  const double* mu = d.mu[m];
  double s2 = 0.0, best = -1.0, bestv = 0.0;
  int besti = -1;
  for (int i = i0 + tid; i < i1; i += FT) {
    double f = 0.0;
    for (int y = 0; y < rm; ++y) f += U[i + (size_t)y * d.ldu[m]] * S.gvec[y];
    double yv = 0.0;
    for (int x = 0; x < pm; ++x) yv += Qm[i + (size_t)x * d.ldq[m]] * S.cvec[x];
    const double val = f / (mu[i] + lab) - yv;
    if (!isfinite(val)) S.bad = 1;
    e_out[i] = val;
    v_out[i] = val;
    s2 += val * val;
    const double av = fabs(val);
    if (av > best) { best = av; bestv = val; besti = i; }
  }
  block_reduce(S.red, s2, best, bestv, besti);
  if (tid == 0) {
    S.ps = S.red.s[0];
    S.pa = S.red.a[0];
    S.pv = S.red.v[0];
    S.pi = S.red.i[0];
    if (S.bad) d.st->status = LR_ENONFINITE;
  }
  cl.sync();
  if (tid < 32) {
    // lane r < SCS reads rank r's partial; then a fixed tree over the lanes
    // (rank order: the chunks of lower ranks hold the lower indices)
    double ps = 0.0, ar = -1.0, vr = 0.0;
    int ir = -1;
    if (lane < SCS) {
      ps = *cl.map_shared_rank(&S.ps, lane);
      ar = *cl.map_shared_rank(&S.pa, lane);
      vr = *cl.map_shared_rank(&S.pv, lane);
      ir = *cl.map_shared_rank(&S.pi, lane);
    }
    for (int o = 1; o < SCS; o <<= 1) {
      const double ps2 = __shfl_down_sync(0xffffffffu, ps, o);
      const double a2 = __shfl_down_sync(0xffffffffu, ar, o);
      const double v2 = __shfl_down_sync(0xffffffffu, vr, o);
      const int i2 = __shfl_down_sync(0xffffffffu, ir, o);
      if ((lane & (2 * o - 1)) == 0) {
        ps += ps2;
        if (a2 > ar || (a2 == ar && i2 >= 0 && (ir < 0 || i2 < ir))) { ar = a2; vr = v2; ir = i2; }
      }
    }
    if (lane == 0) {
      *nrm2 = ps;
      *amax = ir >= 0 ? ir : 0;
      *vmax = vr;
    }
  }
  cl.sync();  // partials and items read before the next fibre overwrites them
}

__global__ void __launch_bounds__(FT) t3_search_kernel(T3Dev d) {
  __shared__ SearchSmem S;
  cg::cluster_group cl = cg::this_cluster();
  if (d.st->done || d.st->status) return;  // the same for every CTA of the cluster
  const int rank = (int)cl.block_rank();
  if (threadIdx.x < 3) S.pos[threadIdx.x] = d.st->pos[threadIdx.x];
  __syncthreads();
  const int seq[8] = {1, 2, 0, 1, 2, 0, 1, 2};
  for (int t = 0; t < 8; ++t) {
    const int m = seq[t];
    int oa, ob;
    other_modes(m, oa, ob);
    double nrm2 = 0.0, v = 0.0;
    int a2 = 0;
    cluster_fibre(d, S, cl, m, S.pos[oa], S.pos[ob], d.e[m], d.v[m], &nrm2, &a2, &v);
    if (threadIdx.x == 0) {
      if (rank == 0) {
        d.st->fnrm2[m] = nrm2;
        d.st->fval[m] = v;
      }
      if (t < 6) S.pos[m] = a2;
    }
    __syncthreads();
  }
  if (rank == 0 && threadIdx.x < 3) d.st->pos[threadIdx.x] = S.pos[threadIdx.x];
}

// Probe fibres from a job list (mode, a, b): square norm and argmax of each.
__global__ void __launch_bounds__(FT) t3_probe_kernel(T3Dev d, const int* __restrict__ jobs, double* __restrict__ nrm2,
                                                        int* __restrict__ amax) {
  __shared__ FibreSmem S;
  const int f = blockIdx.x;
  const int m = jobs[3 * f], a = jobs[3 * f + 1], b = jobs[3 * f + 2];
  double v = 0.0;
  t3_fibre(d, S, m, a, b, nullptr, nullptr, nullptr, &nrm2[f], &amax[f], &v);
}

// Pivot of the step: rho = R(i, j, k), the first pivot's size, and whether
// this one is negligible (no basis update).
__global__ void t3_pivot_kernel(T3Dev d) {
  T3State* s = d.st;
  if (s->done || s->status) return;
  const double rho = s->fval[0];
  s->rho = rho;
  s->steps += 1;
  if (s->rho0 < 0.0) {
    s->rho0 = fabs(rho);
    if (s->rho0 == 0.0) { s->done = 1; s->converged = 1; }
  }
  s->negl = (s->done || fabs(rho) <= 1e-14 * s->rho0) ? 1 : 0;
  for (int m = 0; m < 3; ++m) s->add[m] = s->negl ? 0 : (s->p[m] < T3P ? 1 : 0);
}

// h[m][j] = Q_m(:, j) . v_m (CTA (j, m), j < p_m).
__global__ void __launch_bounds__(FT) t3_dots_kernel(T3Dev d) {
  __shared__ RedSmem R;
  const int j = blockIdx.x, m = blockIdx.y;
  if (d.st->done || d.st->status || !d.st->add[m] || j >= d.st->p[m]) return;
  const double* q = d.Q[m] + (size_t)j * d.ldq[m];
  const double* v = d.v[m];
  double s = 0.0;
  for (int i = threadIdx.x; i < d.n[m]; i += FT) s += q[i] * v[i];
  block_reduce(R, s, 0.0, 0.0, -1);
  if (threadIdx.x == 0) d.h[m][j] = R.s[0];
}

// v_m <- v_m - Q_m h_m.
__global__ void t3_axpy_kernel(T3Dev d) {
  const int m = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (d.st->done || d.st->status || !d.st->add[m] || i >= d.n[m]) return;
  const int p = d.st->p[m];
  double acc = 0.0;
  for (int j = 0; j < p; ++j) acc += d.Q[m][i + (size_t)j * d.ldq[m]] * d.h[m][j];
  d.v[m][i] -= acc;
}

// Normalise v_m into column p_m of Q_m (or drop the fibre if its orthogonal
// part is below 1e-13 of it), and y_m = M_m Q_m(I_m, p_m).
__global__ void __launch_bounds__(FT) t3_addbasis_kernel(T3Dev d) {
  __shared__ RedSmem R;
  __shared__ double qI[T3P];
  const int m = blockIdx.x, tid = threadIdx.x;
  if (d.st->done || d.st->status || !d.st->add[m]) return;
  const int n = d.n[m], p = d.st->p[m];
  double s = 0.0;
  for (int i = tid; i < n; i += FT) s += d.v[m][i] * d.v[m][i];
  block_reduce(R, s, 0.0, 0.0, -1);
  const double nv2 = R.s[0];
  const double ne2 = d.st->fnrm2[m];
  if (!(ne2 > 0.0) || !(nv2 > 1e-26 * ne2)) {
    if (tid == 0) d.st->add[m] = 0;
    return;
  }
  const double sc = 1.0 / sqrt(nv2);
  double* qn = d.Q[m] + (size_t)p * d.ldq[m];
  for (int i = tid; i < n; i += FT) qn[i] = d.v[m][i] * sc;
  __syncthreads();
  for (int x = tid; x < p; x += FT) qI[x] = qn[d.I[m][x]];
  __syncthreads();
  for (int r = tid; r < p; r += FT) {
    double acc = 0.0;
    for (int x = 0; x < p; ++x) acc += d.Minv[m][r + (size_t)x * T3P] * qI[x];
    d.y[m][r] = acc;
  }
}

// DEIM residual of the new basis vector: v_m = q - Q_m(:, :p) y_m, zero on I_m.
__global__ void t3_deimres_kernel(T3Dev d) {
  const int m = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (d.st->done || d.st->status || !d.st->add[m] || i >= d.n[m]) return;
  const int p = d.st->p[m];
  if (d.inI[m][i]) { d.v[m][i] = 0.0; return; }
  double acc = d.Q[m][i + (size_t)p * d.ldq[m]];
  for (int x = 0; x < p; ++x) acc -= d.Q[m][i + (size_t)x * d.ldq[m]] * d.y[m][x];
  d.v[m][i] = acc;
}

// New DEIM index (largest |residual| outside I_m, lowest on ties), bordered
// update of M_m = Q_m(I_m, :)^-1, and p_m + 1.
__global__ void __launch_bounds__(FT) t3_deimpick_kernel(T3Dev d) {
  __shared__ RedSmem R;
  __shared__ double z[T3P];
  const int m = blockIdx.x, tid = threadIdx.x;
  if (d.st->done || d.st->status || !d.st->add[m]) return;
  const int n = d.n[m], p = d.st->p[m];
  double best = -1.0, bv = 0.0;
  int bi = -1;
  for (int i = tid; i < n; i += FT) {
    if (d.inI[m][i]) continue;
    const double a = fabs(d.v[m][i]);
    if (a > best) { best = a; bv = d.v[m][i]; bi = i; }
  }
  block_reduce(R, 0.0, best, bv, bi);
  const int inew = R.i[0];
  const double sres = R.v[0];
  if (inew < 0 || !(sres != 0.0) || !isfinite(sres)) {
    if (tid == 0) d.st->add[m] = 0;
    return;
  }
  // z^T = Q_m(inew, :p) M_m
  double* M = d.Minv[m];
  for (int c = tid; c < p; c += FT) {
    double acc = 0.0;
    for (int x = 0; x < p; ++x) acc += d.Q[m][inew + (size_t)x * d.ldq[m]] * M[x + (size_t)c * T3P];
    z[c] = acc;
  }
  __syncthreads();
  const double is = 1.0 / sres;
  const double* y = d.y[m];
  for (int w = tid; w < p * p; w += FT) {
    const int r = w % p, c = w / p;
    M[r + (size_t)c * T3P] += y[r] * z[c] * is;
  }
  for (int r = tid; r < p; r += FT) {
    M[r + (size_t)p * T3P] = -y[r] * is;
    M[p + (size_t)r * T3P] = -z[r] * is;
  }
  if (tid == 0) {
    M[p + (size_t)p * T3P] = is;
    d.I[m][p] = inew;
    d.inI[m][inew] = 1;
    d.st->p[m] = p + 1;
  }
}

// out = in x_mode A: out[.., i, ..] = sum_{x < K} A(i, x) in[.., x, ..] with
// A(i, x) = A[rowmap(i) * ars + x * acs] (rowmap null: i); optionally divided
// by mu0[I0[x0]] + mu1[I1[x1]] + mu2[I2[x2]].
// A negative dimension -1 - k (od or K) stands for the basis size p_k of the
// state; with skip_negl the product is not formed on a step whose pivot was
// negligible (the core is unchanged).
__global__ void t3_modeprod_kernel(T3ModeProd a, T3Dev d) {
  const T3State* s = d.st;
  if (s->status || (a.skip_negl && (s->negl || s->done))) return;
  int od[3];
  for (int k = 0; k < 3; ++k) od[k] = a.od[k] >= 0 ? a.od[k] : s->p[-1 - a.od[k]];
  const int K = a.K >= 0 ? a.K : s->p[-1 - a.K];
  const size_t total = (size_t)od[0] * od[1] * od[2];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
  const int x0 = (int)(t % od[0]);
  const int x1 = (int)((t / od[0]) % od[1]);
  const int x2 = (int)(t / ((size_t)od[0] * od[1]));
  const int xo[3] = {x0, x1, x2};
  const int i = xo[a.mode];
  size_t base = 0;
  for (int k = 0; k < 3; ++k)
    if (k != a.mode) base += (size_t)xo[k] * a.is[k];
  const size_t arow = (size_t)(a.rowmap ? a.rowmap[i] : i) * a.ars;
  double acc = 0.0;
  for (int x = 0; x < K; ++x) acc += a.A[arow + (size_t)x * a.acs] * a.in[base + (size_t)x * a.is[a.mode]];
  if (a.divlam) acc /= d.mu[0][d.I[0][x0]] + d.mu[1][d.I[1][x1]] + d.mu[2][d.I[2][x2]];
  a.out[(size_t)x0 * a.os[0] + (size_t)x1 * a.os[1] + (size_t)x2 * a.os[2]] = acc;
  }
}

// End of a step: ||C||_F, the step test, and the next search start (the
// largest |e_1| outside I_1, with the last j, k).
__global__ void __launch_bounds__(FT) t3_decide_kernel(T3Dev d, double tol) {
  __shared__ RedSmem R;
  T3State* s = d.st;
  if (s->done || s->status) return;
  const int tid = threadIdx.x;
  const int p0 = s->p[0], p1 = s->p[1], p2 = s->p[2];
  double c2 = 0.0;
  for (int w = tid; w < p0 * p1 * p2; w += FT) {
    const int x0 = w % p0, x1 = (w / p0) % p1, x2 = w / (p0 * p1);
    const double c = d.C[x0 + (size_t)T3P * (x1 + (size_t)T3P * x2)];
    c2 += c * c;
  }
  double best = -1.0, bv = 0.0;
  int bi = -1;
  if (!s->negl)
    for (int i = tid; i < d.n[0]; i += FT) {
      if (d.inI[0][i]) continue;
      const double a = fabs(d.e[0][i]);
      if (a > best) { best = a; bv = d.e[0][i]; bi = i; }
    }
  block_reduce(R, c2, best, bv, bi);
  if (tid == 0) {
    const double nC = sqrt(R.s[0]);
    s->nrmC = nC;
    if (s->negl) {
      s->small = 2;
    } else {
      const double upd = sqrt(s->fnrm2[0]) * sqrt(s->fnrm2[1]) * sqrt(s->fnrm2[2]) / (s->rho * s->rho);
      s->upd = upd;
      s->small = upd <= tol * nC ? s->small + 1 : 0;
      s->pos[0] = R.i[0] >= 0 ? R.i[0] : 0;
    }
  }
}

// Probe round: the estimates of ||R||_F from the random fibres (mean square
// norm times the number of fibres of the mode) and from the cross fibres
// (root of the sum), the largest fibre (first in job order on ties), and the
// decision.  counts: random and cross fibres of each mode, in job order.
// One CTA; every sum is a fixed-order block reduction.
__global__ void __launch_bounds__(FT) t3_probe_reduce_kernel(T3Dev d, const int* __restrict__ jobs,
                                                               const double* __restrict__ nrm2,
                                                               const int* __restrict__ amax, T3ProbeCounts cnt,
                                                               double tol) {
  __shared__ RedSmem R;
  __shared__ double est;
  const int tid = threadIdx.x;
  T3State* s = d.st;
  if (tid == 0) est = 0.0;
  int f0 = 0;
  for (int seg = 0; seg < 6; ++seg) {
    const int m = seg / 2;
    const int len = (seg & 1) ? cnt.ncross[m] : cnt.nrand[m];
    double acc = 0.0;
    for (int f = f0 + tid; f < f0 + len; f += FT) acc += nrm2[f];
    block_reduce(R, acc, 0.0, 0.0, -1);
    if (tid == 0 && len > 0) {
      int oa, ob;
      other_modes(m, oa, ob);
      const double e = (seg & 1) ? sqrt(R.s[0]) : sqrt(R.s[0] * (double)d.n[oa] * (double)d.n[ob] / len);
      est = fmax(est, e);
    }
    __syncthreads();
    f0 += len;
  }
  double best = -1.0;
  int bi = -1;
  for (int f = tid; f < f0; f += FT)
    if (nrm2[f] > best) { best = nrm2[f]; bi = f; }
  block_reduce(R, 0.0, best, 0.0, bi);
  if (tid != 0) return;
  const int wf = R.i[0];
  s->est = est;
  s->probe_rounds += 1;
  if (est <= tol * s->nrmC) {
    s->done = 1;
    s->converged = 1;
    return;
  }
  s->small = 0;
  if (wf >= 0) {
    const int m = jobs[3 * wf];
    int oa, ob;
    other_modes(m, oa, ob);
    s->pos[oa] = jobs[3 * wf + 1];
    s->pos[ob] = jobs[3 * wf + 2];
    s->pos[m] = amax[wf];
  }
}

// A = C_(m)^T: rows (xa + pa xb) over the other two modes, column xm.
__global__ void t3_unfold_kernel(T3Dev d, int m, double* __restrict__ A, int lda) {
  int oa, ob;
  other_modes(m, oa, ob);
  const int pm = d.st->p[m], pa = d.st->p[oa], pb = d.st->p[ob];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pm * pa * pb) return;
  const int row = t % (pa * pb), xm = t / (pa * pb);
  const int xa = row % pa, xb = row / pa;
  int x[3];
  x[m] = xm;
  x[oa] = xa;
  x[ob] = xb;
  A[row + (size_t)xm * lda] = d.C[x[0] + (size_t)T3P * (x[1] + (size_t)T3P * x[2])];
}

}  // namespace

__global__ void t3_widen_kernel(const float* __restrict__ in, double* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

#define T3_LAUNCH_CHECK() return cudaGetLastError()

cudaError_t launch_t3_widen(const float* in, double* out, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  t3_widen_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_search(const T3Dev& d, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(SCS, 1, 1);
  cfg.blockDim = dim3(FT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = SCS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, t3_search_kernel, d);
}

cudaError_t launch_t3_probe(const T3Dev& d, int nfib, const int* jobs, double* nrm2, int* amax, cudaStream_t st) {
  if (nfib <= 0) return cudaSuccess;
  t3_probe_kernel<<<nfib, FT, 0, st>>>(d, jobs, nrm2, amax);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_pivot(const T3Dev& d, cudaStream_t st) {
  t3_pivot_kernel<<<1, 1, 0, st>>>(d);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_basis_update(const T3Dev& d, int nmax, cudaStream_t st) {
  const dim3 dots(T3P, 3), rows((nmax + 255) / 256, 3);
  for (int pass = 0; pass < 2; ++pass) {  // two passes of classical Gram-Schmidt
    t3_dots_kernel<<<dots, FT, 0, st>>>(d);
    t3_axpy_kernel<<<rows, 256, 0, st>>>(d);
  }
  t3_addbasis_kernel<<<3, FT, 0, st>>>(d);
  t3_deimres_kernel<<<rows, 256, 0, st>>>(d);
  t3_deimpick_kernel<<<3, FT, 0, st>>>(d);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_modeprod(const T3ModeProd& a, const T3Dev& d, cudaStream_t st) {
  size_t total = 1;  // upper bound: a basis size is at most T3P
  for (int k = 0; k < 3; ++k) total *= (size_t)(a.od[k] >= 0 ? a.od[k] : T3P);
  if (total == 0) return cudaSuccess;
  // grid-stride over a grid of at most 256 CTAs (the sizes read on the device
  // are usually far below the bound)
  const size_t blocks = std::min<size_t>((total + 255) / 256, 256);
  t3_modeprod_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, d);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_decide(const T3Dev& d, double tol, cudaStream_t st) {
  t3_decide_kernel<<<1, FT, 0, st>>>(d, tol);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_probe_reduce(const T3Dev& d, const int* jobs, const double* nrm2, const int* amax,
                                   const T3ProbeCounts& c, double tol, cudaStream_t st) {
  t3_probe_reduce_kernel<<<1, FT, 0, st>>>(d, jobs, nrm2, amax, c, tol);
  T3_LAUNCH_CHECK();
}

cudaError_t launch_t3_unfold(const T3Dev& d, int m, int total, double* A, int lda, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  t3_unfold_kernel<<<(total + 255) / 256, 256, 0, st>>>(d, m, A, lda);
  T3_LAUNCH_CHECK();
}

}  // namespace lrp
