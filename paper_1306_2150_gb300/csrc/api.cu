// C ABI of liblrpoisson.so: handle, plan cache, workspace and the entry points
// declared in include/lrpoisson.h.  Every numerical step runs in the kernels of
// dst.cu, cross.cu and core.cu; this file validates arguments, lays out the
// workspace and enqueues the launches on the handle's stream.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <initializer_list>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lr_internal.h"
#include "maxvol.h"

using namespace lrp;

struct lr_handle_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  std::map<int, std::unique_ptr<Plan>> plans;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  SolveState* h_state = nullptr;  // pinned
  int* h_piv = nullptr;           // pinned, 2 * KMAX
  double* h_w = nullptr;          // pinned, 2 * KMAX (weights read back by refinement)
  lr_info info{};
  int last_kcap = 0;
  cudaEvent_t ev[LR_NUM_PHASES + 1] = {};
  bool timed = false;
  // batched solves: internal streams, fork/join events, pinned status array
  cudaStream_t bstreams[32] = {};
  cudaEvent_t bjoin[32] = {};
  cudaEvent_t bfork = nullptr;
  SolveState* h_bstate = nullptr;
  int bstate_cap = 0;
  // captured CUDA graphs (LR_FLAG_GRAPH), keyed by every pointer and size
  cudaStream_t cap_stream = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  unsigned long long ws_gen = 0;
  int last_cs = 0;
  // float64 buffers of iterative refinement (solution, correction, residual)
  void* ws2 = nullptr;
  size_t ws2_bytes = 0;
  // workspace of full-grid solves (two m x m buffers and the transform scratch)
  void* ws3 = nullptr;
  size_t ws3_bytes = 0;
  // Stokes workspace and a pinned buffer for its Gram matrices
  void* ws4 = nullptr;
  size_t ws4_bytes = 0;
  double* h_big = nullptr;
  // workspace of 3D Tucker solves
  void* ws5 = nullptr;
  size_t ws5_bytes = 0;
  // autotuned cluster sizes of single solves, keyed (m, precision, operator),
  // and indices per cross CTA of batched solves, per precision
  std::map<std::tuple<int, int, int>, int> tuned_cs;
  int batch_ipc[2] = {2048, 2048};
  // phase-batched solves: twiddle tables of length 4096 (float64, float32),
  // the device copy of the last batch's descriptors and its pinned staging
  // buffer (reused once the event says the previous upload has run), and one
  // device descriptor block per captured graph
  void* tw4096[2] = {nullptr, nullptr};
  char* bdesc = nullptr;
  size_t bdesc_cap = 0;
  char* h_bdesc = nullptr;
  size_t h_bdesc_cap = 0;
  cudaEvent_t bdesc_ev = nullptr;
  std::map<std::string, char*> graph_desc;
  int cross_rows[2] = {4096, 4096};  // indices per CTA of the batched cross (float64, float32)
  int last_batch = 0;                // problems of the last lr_poisson2d_batched call (status record)
  int dst_fused[2] = {0, 1};         // batched transforms of M > 4096: one pass per column (1, float32
                                     // only) or the four-step passes through scratch (0); float64
                                     // keeps the four-step passes (FP64-bound either way, and faster)
  size_t ws_limit = 0;               // cap on the workspaces' total bytes (0: none)
};

namespace {

// NVTX range on the calling thread (profilers attribute the kernels launched
// inside it; a no-op without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Consecutive phases of one call: to() closes the open phase and opens the
// next; the last one closes on scope exit (early returns included).
struct NvtxPhase {
  bool open = false;
  void to(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhase() {
    if (open) nvtxRangePop();
  }
};

lr_status fail(lr_handle h, lr_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

lr_status cuda_fail(lr_handle h, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, LR_ECUDA, msg);
}

#define LR_CUDA(h, call, where)                     \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

const char* const kNonFiniteMsg =
    "non-finite value in the rounding core (in LR_MIXED: frequency-space entries outside the float32 range)";

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
int round_up(int x, int a) { return (x + a - 1) / a * a; }

lr_status get_plan(lr_handle h, int m, Plan** out) {
  auto it = h->plans.find(m);
  if (it != h->plans.end()) { *out = it->second.get(); return LR_OK; }
  std::unique_ptr<Plan> p(new Plan());
  std::string e = build_plan(m, *p);
  if (!e.empty()) return fail(h, LR_ENOMEM, e);
  *out = p.get();
  h->plans[m] = std::move(p);
  return LR_OK;
}

// Grow one of the handle's workspaces to `need` bytes (freeing the old one
// after the stream has finished with it), within the handle's limit.
lr_status grow_ws(lr_handle h, void** slot, size_t* slot_bytes, size_t need, const char* what) {
  if (need <= *slot_bytes) return LR_OK;
  const size_t total = h->ws_bytes + h->ws2_bytes + h->ws3_bytes + h->ws4_bytes + h->ws5_bytes;
  if (h->ws_limit && total - *slot_bytes + need > h->ws_limit)
    return fail(h, LR_ENOMEM, std::string(what) + ": " + std::to_string(need) +
                                  " bytes would exceed the handle's workspace limit of " + std::to_string(h->ws_limit));
  if (*slot) {
    cudaStreamSynchronize(h->stream);
    cudaFree(*slot);
    *slot = nullptr;
    *slot_bytes = 0;
  }
  if (cudaMalloc(slot, need) != cudaSuccess) {
    cudaGetLastError();
    *slot = nullptr;
    return fail(h, LR_ENOMEM, std::string(what) + ": cudaMalloc of " + std::to_string(need) + " bytes failed");
  }
  *slot_bytes = need;
  return LR_OK;
}

lr_status ensure_ws(lr_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return LR_OK;
  const size_t total = h->ws_bytes + h->ws2_bytes + h->ws3_bytes + h->ws4_bytes + h->ws5_bytes;
  if (h->ws_limit && total - h->ws_bytes + bytes > h->ws_limit)
    return fail(h, LR_ENOMEM, "workspace: " + std::to_string(bytes) +
                                  " bytes would exceed the handle's workspace limit of " + std::to_string(h->ws_limit));
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  ++h->ws_gen;  // captured graphs point into the old workspace
  if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LR_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " workspace bytes failed");
  }
  h->ws_bytes = bytes;
  return LR_OK;
}

// Bump allocator over the workspace.
struct Carve {
  size_t off = 0;
  char* base = nullptr;
  template <typename P>
  P* take(size_t bytes) {
    P* p = reinterpret_cast<P*>(base ? base + off : nullptr);
    off += align256(bytes);
    return p;
  }
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

lr_status check_problem(lr_handle h, const lr_mat* rhs, const lr_mat* sol) {
  if (!rhs || !sol) return fail(h, LR_EINVAL, "null rhs or sol");
  const int m = rhs->n1;
  if (m < 1 || rhs->n2 != m) return fail(h, LR_EINVAL, "rhs must be square (n1 == n2 >= 1)");
  if (rhs->r < 1 || rhs->r > KMAX) return fail(h, LR_EINVAL, "rhs->r must be in [1, 64]");
  if (rhs->ld < m || sol->ld < m) return fail(h, LR_EINVAL, "leading dimension smaller than m");
  if (sol->n1 != m || sol->n2 != m) return fail(h, LR_EINVAL, "sol must be m x m");
  if (sol->rmax < 1) return fail(h, LR_EINVAL, "sol->rmax must be >= 1");
  if (rhs->s) return fail(h, LR_EINVAL, "rhs->s must be NULL (fold weights into U)");
  if (!rhs->U || !rhs->V || !sol->U || !sol->V || !sol->s) return fail(h, LR_EINVAL, "null factor pointer");
  if (!aligned16(rhs->U) || !aligned16(rhs->V) || !aligned16(sol->U) || !aligned16(sol->V) || !aligned16(sol->s))
    return fail(h, LR_EINVAL, "factor pointers must be 16-byte aligned");
  if (m > 131072) return fail(h, LR_EINVAL, "m too large (max 131072)");
  return LR_OK;
}

lr_status check_opts(lr_handle h, const lr_options& o) {
  if (o.prec != LR_FP64 && o.prec != LR_MIXED) return fail(h, LR_EINVAL, "unknown precision");
  if (o.op != LR_OP_5PT && o.op != LR_OP_SEMISTAGGERED) return fail(h, LR_EINVAL, "unknown operator");
  if (!(o.eps > 0.0) || !std::isfinite(o.eps) || o.eps >= 1.0) return fail(h, LR_EINVAL, "eps must be in (0, 1)");
  if (o.rmax < 1 || o.rmax > KMAX) return fail(h, LR_EINVAL, "opt->rmax must be in [1, 64]");
  if (!(o.aca_tol_factor > 0.0) || !std::isfinite(o.aca_tol_factor))
    return fail(h, LR_EINVAL, "aca_tol_factor must be positive");
  if (o.probes < 0 || o.probes > 32) return fail(h, LR_EINVAL, "probes must be in [0, 32]");
  if (o.cluster_size < 0 || o.cluster_size > 16) return fail(h, LR_EINVAL, "cluster_size must be in [0, 16]");
  if (o.refine < -1 || o.refine > 8) return fail(h, LR_EINVAL, "refine must be in [-1, 8]");
  return LR_OK;
}

// Geometry of one solve and its workspace slice.
struct SolveGeom {
  int m = 0, r = 0, kcap = 0, ldw = 0, ncap_out = 0, cols_fft = 0;
  size_t M = 0;
  bool four_step = false;
};

SolveGeom geom_of(int m, int r, int sol_rmax, const lr_options& o, const Plan& p) {
  SolveGeom g;
  g.m = m;
  g.r = r;
  g.kcap = o.rmax < m ? o.rmax : m;
  g.ldw = round_up(m, 32);
  g.ncap_out = g.kcap < sol_rmax ? g.kcap : sol_rmax;
  g.M = (size_t)1 << p.logM;
  g.cols_fft = (2 * r > 2 * g.kcap) ? 2 * r : 2 * g.kcap;
  g.four_step = g.M > (size_t)kSmallM;
  return g;
}

template <typename T>
struct Slice {
  T *Uh, *Vh, *C, *R, *Tc, *Tr;
  void* work;
  double *GC, *GR, *d;
  int *I, *J;
};

template <typename T>
Slice<T> carve_slice(Carve& cv, const SolveGeom& g) {
  Slice<T> w;
  w.Uh = cv.template take<T>(sizeof(T) * g.ldw * g.r);
  w.Vh = cv.template take<T>(sizeof(T) * g.ldw * g.r);
  w.C = cv.template take<T>(sizeof(T) * g.ldw * g.kcap);
  w.R = cv.template take<T>(sizeof(T) * g.ldw * g.kcap);
  w.work = cv.template take<char>(g.four_step ? sizeof(cpx<T>) * g.M * g.cols_fft : 16);
  w.GC = cv.template take<double>(sizeof(double) * g.kcap * g.kcap);
  w.GR = cv.template take<double>(sizeof(double) * g.kcap * g.kcap);
  w.d = cv.template take<double>(sizeof(double) * g.kcap);
  w.I = cv.template take<int>(sizeof(int) * g.kcap);
  w.J = cv.template take<int>(sizeof(int) * g.kcap);
  w.Tc = cv.template take<T>(sizeof(T) * KMAX * KMAX);
  w.Tr = cv.template take<T>(sizeof(T) * KMAX * KMAX);
  return w;
}

int launches_of(const SolveGeom& g) { return 2 * (g.four_step ? 3 : 1) + 2; }

// Enqueue the steps of one solve (forward DST to inverse DST) on stream stm.  ev (optional) receives the
// phase boundaries.
template <typename T>
cudaError_t enqueue_solve(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options& o, const Plan& plan,
                          const SolveGeom& g, const Slice<T>& w, SolveState* st, cudaStream_t stm,
                          cudaEvent_t* ev, int* used_cs) {
  const bool f32 = sizeof(T) == 4;
  cudaError_t e;
  if ((e = cudaMemsetAsync(st, 0, sizeof(SolveState), stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], stm)) != cudaSuccess) return e;
  NvtxPhase phase;
  // Forward DST of both factors.
  phase.to("lr:forward_dst");
  ColumnSet fw;
  fw.in[0] = rhs->U; fw.in[1] = rhs->V;
  fw.ld_in[0] = rhs->ld; fw.ld_in[1] = rhs->ld;
  fw.out[0] = w.Uh; fw.out[1] = w.Vh;
  fw.ld_out[0] = g.ldw; fw.ld_out[1] = g.ldw;
  fw.ncol[0] = g.r; fw.ncol[1] = g.r;
  if ((e = launch_dst<T>(plan, fw, IoType::F64, IoType::WORK, w.work, h->num_sms, stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], stm)) != cudaSuccess) return e;
  // Cross approximation in frequency space (symbol, pivots, skeleton).
  phase.to("lr:cross");
  CrossArgs<T> ca;
  ca.m = g.m; ca.r = g.r; ca.kcap = g.kcap; ca.ld = g.ldw;
  ca.Uh = w.Uh; ca.Vh = w.Vh; ca.C = w.C; ca.R = w.R;
  ca.a = f32 ? reinterpret_cast<const T*>(plan.sym_a32[o.op]) : reinterpret_cast<const T*>(plan.sym_a64[o.op]);
  ca.b = f32 ? reinterpret_cast<const T*>(plan.sym_b32[o.op]) : reinterpret_cast<const T*>(plan.sym_b64[o.op]);
  ca.d = w.d; ca.I = w.I; ca.J = w.J; ca.GC = w.GC; ca.GR = w.GR; ca.st = st;
  ca.tol = o.aca_tol_factor * o.eps;
  ca.probes = o.probes;
  ca.seed = o.seed;
  ca.max_probe_rounds = 4;
  ca.max_zero_rows = 16;
  if ((e = launch_cross<T>(ca, o.cluster_size, stm, used_cs)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], stm)) != cudaSuccess) return e;
  // Rounding core.
  phase.to("lr:rounding");
  CoreArgs<T> co;
  co.GC = w.GC; co.GR = w.GR; co.ldg = g.kcap; co.d = w.d;
  co.k_dev = &st->k; co.k_host = 0;
  co.eps = o.eps; co.rmax_out = g.ncap_out;
  co.Tc = w.Tc; co.Tr = w.Tr; co.s_out = sol->s; co.st = st;
  if ((e = launch_core<T>(co, f32, stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], stm)) != cudaSuccess) return e;
  // Inverse DST of the kept columns into the caller's float64 factors;
  phase.to("lr:inverse_dst");
  // the rotation of the skeleton by Tc, Tr (the last step of the rounding) is
  // applied as the transform loads its input.
  ColumnSet iv;
  iv.in[0] = w.C; iv.in[1] = w.R;
  iv.tm[0] = w.Tc; iv.tm[1] = w.Tr;
  iv.k_dev = &st->k;
  iv.ld_in[0] = g.ldw; iv.ld_in[1] = g.ldw;
  iv.out[0] = sol->U; iv.out[1] = sol->V;
  iv.ld_out[0] = sol->ld; iv.ld_out[1] = sol->ld;
  iv.ncol[0] = g.ncap_out; iv.ncol[1] = g.ncap_out;
  iv.dyn_count = &st->rank;
  if ((e = launch_dst<T>(plan, iv, IoType::ROT, IoType::F64, w.work, h->num_sms, stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[4], stm)) != cudaSuccess) return e;
  return cudaSuccess;
}

lr_status ensure_events(lr_handle h) {
  for (auto& e : h->ev)
    if (!e && cudaEventCreate(&e) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "event create");
  return LR_OK;
}

// Run `body` (which enqueues work on the stream it is given) either directly
// on the handle's stream, or -- with LR_FLAG_GRAPH -- through a CUDA graph
// captured once per key on an internal stream and replayed on the handle's
// stream.  Graphs bake in every pointer, so the key holds all of them and
// the workspace generation.
template <typename F>
lr_status run_maybe_graph(lr_handle h, bool graph, const std::string& key, F&& body) {
  if (!graph) {
    cudaError_t e = body(h->stream);
    return e == cudaSuccess ? LR_OK : cuda_fail(h, e, "enqueue");
  }
  const std::string k = key + "|ws" + std::to_string(h->ws_gen);
  auto it = h->graphs.find(k);
  if (it == h->graphs.end()) {
    if (!h->cap_stream) LR_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream");
    LR_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = body(h->cap_stream);
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      return cuda_fail(h, e != cudaSuccess ? e : e2, "graph capture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    if (h->graphs.size() >= 32) {  // bounded cache
      cudaStreamSynchronize(h->stream);
      for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
      h->graphs.clear();
      for (auto& kv : h->graph_desc) cudaFree(kv.second);
      h->graph_desc.clear();
    }
    it = h->graphs.emplace(k, ex).first;
  }
  LR_CUDA(h, cudaGraphLaunch(it->second, h->stream), "graph launch");
  return LR_OK;
}

std::string key_of(const char* tag, const lr_mat* a, int n, const lr_mat* b, const lr_options& o) {
  std::string k(tag);
  char buf[256];
  for (int i = 0; i < n; ++i) {
    snprintf(buf, sizeof buf, "|%d,%d,%d,%d,%p,%p,%p;%d,%d,%p,%p,%p", a[i].n1, a[i].r, a[i].rmax, a[i].ld,
             (void*)a[i].U, (void*)a[i].s, (void*)a[i].V, b[i].rmax, b[i].ld, (void*)b[i].U, (void*)b[i].s,
             (void*)b[i].V);
    k += buf;
  }
  snprintf(buf, sizeof buf, "|o%d,%d,%.17g,%d,%.17g,%d,%llu,%u,%d", (int)o.prec, (int)o.op, o.eps, o.rmax,
           o.aca_tol_factor, o.probes, o.seed, o.flags & ~(unsigned)(LR_FLAG_ASYNC | LR_FLAG_TIMING),
           o.cluster_size);
  k += buf;
  return k;
}

template <typename T>
lr_status solve2d(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options& o, Plan* plan) {
  const SolveGeom g = geom_of(rhs->n1, rhs->r, sol->rmax, o, *plan);
  Carve c;
  carve_slice<T>(c, g);
  const size_t st_off = c.off;
  c.take<SolveState>(sizeof(SolveState));
  lr_status s = ensure_ws(h, c.off);
  if (s != LR_OK) return s;
  Carve c2;
  c2.base = static_cast<char*>(h->ws);
  const Slice<T> w = carve_slice<T>(c2, g);
  SolveState* st = reinterpret_cast<SolveState*>(static_cast<char*>(h->ws) + st_off);
  const bool timing = (o.flags & LR_FLAG_TIMING) != 0;
  const bool graph = (o.flags & LR_FLAG_GRAPH) != 0 && !timing;
  if (timing && (s = ensure_events(h)) != LR_OK) return s;
  h->timed = timing;
  int used_cs = 0;
  // transform variant for this call (restored on return)
  const int pi = sizeof(T) == 4 ? 1 : 0;
  struct Restore { Plan* p; int i, v; ~Restore() { p->use_cluster[i] = v; } } restore{plan, pi, plan->use_cluster[pi]};
  if (o.flags & LR_FLAG_CLUSTER_DST) plan->use_cluster[pi] = 1;
  s = run_maybe_graph(h, graph, key_of("single", rhs, 1, sol, o), [&](cudaStream_t stm) -> cudaError_t {
    cudaError_t e = enqueue_solve<T>(h, rhs, sol, o, *plan, g, w, st, stm, timing ? h->ev : nullptr, &used_cs);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h->h_state, st, sizeof(SolveState), cudaMemcpyDeviceToHost, stm)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(h->h_piv, w.I, sizeof(int) * g.kcap, cudaMemcpyDeviceToHost, stm)) != cudaSuccess)
      return e;
    return cudaMemcpyAsync(h->h_piv + KMAX, w.J, sizeof(int) * g.kcap, cudaMemcpyDeviceToHost, stm);
  });
  if (s != LR_OK) return s;
  h->info.launches = launches_of(g);
  if (used_cs) h->last_cs = used_cs;   // a replayed graph launches nothing from the host
  h->info.cluster_size = h->last_cs;
  h->last_kcap = g.kcap;
  if (o.flags & LR_FLAG_ASYNC) return LR_OK;
  LR_CUDA(h, cudaStreamSynchronize(h->stream), "solve");
  const SolveState& hs = *h->h_state;
  sol->r = hs.rank;
  if (hs.status) return fail(h, static_cast<lr_status>(hs.status), kNonFiniteMsg);
  if (!hs.converged) return fail(h, LR_ENOCONV, "cross did not converge within opt->rmax steps");
  if (hs.cut) return fail(h, LR_ENOCONV, "solution rank exceeds sol->rmax; result truncated");
  return LR_OK;
}

// Mixed-precision solve followed by up to `rounds` rounds of refinement in
// float64 (residual correction):
//   X  <- solve(F)                        (mixed, at max(eps, 1e-6))
//   repeat: Res = F - A X                 (exact, low rank r + 2R, float64)
//           Res <- QR-round(Res, 1e-8)    (shifted Cholesky QR + core SVD)
//           D   = s0 solve(Res / s0)      (mixed, at 1e-5, at unit scale)
//           X   <- round(X + D, eps)      (float64 rounding, Section 3)
//   until the error estimate sigma_0(D) / sigma_0(X) * (ratio of successive
//   corrections) is below eps / 2, or the corrections stop shrinking.
// The float32 error of X lives in its factors, so Res stays low rank; each
// round multiplies the error by about the accuracy of the correction solve.
struct RefineBufs {
  double *XU, *XV, *Xs;        // X, with room for X + D (KMAX columns)
  double *L, *Rt, *Lb, *Rb;    // residual factors and Cholesky QR ping-pong buffers
  double *FU, *FV;             // rounded residual (partial sums over chunks of X)
  double *G0, *G1, *T0, *T1, *Ra0, *Ra1, *Tc, *Tr, *rs, *part;
  int* qout;
  SolveState* st;
  double* aux;  // 4 KMAX scratch values (quadrature nodes, weights)
};

void carve_refine(Carve& c, RefineBufs& b, int ld, int m) {
  const size_t col = sizeof(double) * (size_t)ld * KMAX;
  const size_t sq = sizeof(double) * KMAX * KMAX;
  b.XU = c.take<double>(col);
  b.XV = c.take<double>(col);
  b.L = c.take<double>(col);
  b.Rt = c.take<double>(col);
  b.Lb = c.take<double>(col);
  b.Rb = c.take<double>(col);
  b.FU = c.take<double>(col);
  b.FV = c.take<double>(col);
  b.Xs = c.take<double>(sizeof(double) * KMAX);
  b.rs = c.take<double>(sizeof(double) * KMAX);
  b.G0 = c.take<double>(sq);
  b.G1 = c.take<double>(sq);
  b.T0 = c.take<double>(sq);
  b.T1 = c.take<double>(sq);
  b.Ra0 = c.take<double>(sq);
  b.Ra1 = c.take<double>(sq);
  b.Tc = c.take<double>(sq);
  b.Tr = c.take<double>(sq);
  b.part = c.take<double>(sq * (size_t)((m + 63) / 64));
  b.qout = c.take<int>(sizeof(int) * 2);
  b.st = c.take<SolveState>(sizeof(SolveState));
  b.aux = c.take<double>(sizeof(double) * 4 * KMAX);
}

constexpr int kQrSteps = 5;
constexpr int kQrShiftedSteps = 3;

// Rounding of L diag(d) Rt^T (q <= 64 columns, d = null: ones) through QR
// factors of L and Rt by shifted Cholesky QR and the SVD of the core
// R_L diag(d) R_R^T (Section 3).  Backward stable, so it keeps a product far
// smaller than its factors (a residual) and returns factors orthonormal to
// working accuracy.  Results (rank K, sigma_0 on the host) go to U, V, s
// (ld ldo); the weights are folded into U if fold is 1 (s) or 2 (s / s_0).
// Scratch: b.L, b.Rt, b.Lb, b.Rb, the small matrices and b.st.
lr_status qr_round(lr_handle h, const RefineBufs& b, const double* Lin, const double* Rin, int ldin, int m, int q,
                   const double* d, double eps, int rmax, double* U, double* V, double* s_out, int ldo, int fold,
                   bool jacobi_fp32, int* K, double* sigma0, double eps_abs = 0.0) {
  cudaStream_t stm = h->stream;
  const int ld = m + (m & 1);
  const double* Xl = Lin;
  const double* Xr = Rin;
  int ldx = ldin;
  // Shift of the first three steps (equilibrated Gram matrix, ||G|| <= q).
  // Each shifted step maps a singular value sigma to sigma / sqrt(sigma^2 +
  // shift) and loses nothing (Q = X R^-1 exactly), so three of them bring a
  // factor of condition beyond 1 / eps64 (columns nearly in the span of the
  // others, as the terms of an exponential sum at neighbouring nodes are)
  // within reach of the two plain steps that make Q orthonormal; no column
  // is ever dropped but an exactly zero one.
  const double shift = 11.0 * ((double)m * q + (double)q * (q + 1)) * (DBL_EPSILON / 2) * q;
  for (int step = 0; step < kQrSteps; ++step) {
    double* Yl = (step & 1) ? b.L : b.Lb;   // ping-pong: Lin -> Lb -> L -> Lb -> L -> Lb
    double* Yr = (step & 1) ? b.Rt : b.Rb;
    LR_CUDA(h, launch_gram(Xl, m, ldx, q, b.G0, q, b.part, h->num_sms, stm), "gram");
    LR_CUDA(h, launch_gram(Xr, m, ldx, q, b.G1, q, b.part, h->num_sms, stm), "gram");
    CholQrArgs a;
    a.G[0] = b.G0; a.G[1] = b.G1;
    a.T[0] = b.T0; a.T[1] = b.T1;
    a.Racc[0] = b.Ra0; a.Racc[1] = b.Ra1;
    a.qout = b.qout;
    a.q = q;
    a.first = step == 0;
    a.shift = step < kQrShiftedSteps ? shift : 0.0;
    a.floor_rel = 0.0;
    LR_CUDA(h, launch_cholqr_step(a, stm), "cholesky qr");
    LR_CUDA(h, (launch_rotate<double, double>(Xl, ldx, m, nullptr, q, b.T0, false, &b.qout[0], Yl, ld, stm)), "qr");
    LR_CUDA(h, (launch_rotate<double, double>(Xr, ldx, m, nullptr, q, b.T1, false, &b.qout[1], Yr, ld, stm)), "qr");
    Xl = Yl;
    Xr = Yr;
    ldx = ld;
  }
  LR_CUDA(h, cudaMemsetAsync(b.st, 0, sizeof(SolveState), stm), "state reset");
  CoreArgs<double> co;
  co.GC = b.Ra0; co.GR = b.Ra1; co.ldg = KMAX; co.d = d;
  co.k_dev = nullptr; co.k_host = q;
  co.eps = eps; co.rmax_out = rmax;
  co.eps_abs = eps_abs;
  co.Tc = b.Tc; co.Tr = b.Tr; co.s_out = s_out; co.st = b.st;
  co.tri_given = 1;
  LR_CUDA(h, launch_core<double>(co, jacobi_fp32, stm), "qr rounding core");
  LR_CUDA(h, (launch_rotate<double, double>(Xl, ld, m, nullptr, q, b.Tc, false, &b.st->rank, U, ldo, stm)), "rot");
  LR_CUDA(h, (launch_rotate<double, double>(Xr, ld, m, nullptr, q, b.Tr, false, &b.st->rank, V, ldo, stm)), "rot");
  if (fold) LR_CUDA(h, launch_fold_weights(m, q, &b.st->rank, U, ldo, s_out, fold == 2, stm), "fold");
  LR_CUDA(h, cudaMemcpyAsync(h->h_state, b.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stm), "state copy");
  LR_CUDA(h, cudaStreamSynchronize(stm), "qr rounding");
  if (h->h_state->status) return fail(h, static_cast<lr_status>(h->h_state->status), kNonFiniteMsg);
  *K = h->h_state->rank;
  *sigma0 = h->h_state->sigma0;
  if (h->h_state->cut) return fail(h, LR_ENOCONV, "rank exceeds rmax; result truncated");
  return LR_OK;
}
constexpr int kQrRoundLaunches = kQrSteps * 7 + 4;

lr_status solve2d_refined(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options& o, Plan* plan,
                          int rounds) {
  const int m = rhs->n1, r = rhs->r;
  const int ld = m + (m & 1);
  RefineBufs b;
  Carve sizing;
  carve_refine(sizing, b, ld, m);
  if (sizing.off > h->ws2_bytes) {
    const lr_status sg = grow_ws(h, &h->ws2, &h->ws2_bytes, sizing.off, "refinement buffers");
    if (sg != LR_OK) return sg;
  }
  Carve cv;
  cv.base = static_cast<char*>(h->ws2);
  carve_refine(cv, b, ld, m);
  cudaStream_t stm = h->stream;
  lr_options o1 = o;
  o1.eps = o.eps > 1e-6 ? o.eps : 1e-6;
  o1.flags = 0;
  o1.refine = -1;
  lr_mat X = {m, m, 0, KMAX, ld, b.XU, b.Xs, b.XV};
  lr_status s = solve2d<float>(h, rhs, &X, o1, plan);
  if (s != LR_OK && s != LR_ENOCONV) return s;
  lr_status worst = s;
  // The first solve's cross statistics and pivots describe the solve.
  const SolveState first = *h->h_state;
  int piv[2 * KMAX];
  std::memcpy(piv, h->h_piv, sizeof piv);
  const int cs_first = h->info.cluster_size;
  int launches = h->info.launches;
  double sigX = first.sigma0, corr = 0.0, prev = 0.0;
  int done = 0;
  for (int it = 0; it < rounds && X.r > 0; ++it) {
    const int R1 = X.r;
    if (R1 >= KMAX) { worst = LR_ENOCONV; fail(h, worst, "no room for the correction (R = 64)"); break; }
    // Res = F - A X accumulated over chunks X_j of X's columns (largest
    // singular values first, where F and A X cancel):
    //   Res_j = round(Res_{j-1} - A X_j),  Res_0 = F,
    // each rounding on at most 64 columns (width of Res_{j-1} + 2 |X_j|).
    const double* FUp = rhs->U;
    const double* FVp = rhs->V;
    int fr = r, fld = rhs->ld, off = 0, Kres = 0;
    double rs0 = 0.0;
    bool stuck = false;
    while (off < R1) {
      const int c = std::min(R1 - off, (KMAX - fr) / 2);
      if (c < 1) { stuck = true; break; }
      const int q = fr + 2 * c;
      const bool last = off + c == R1;
      LR_CUDA(h, launch_residual_factors(m, fr, c, FUp, FVp, fld, X.U + (size_t)off * ld, X.s + off,
                                         X.V + (size_t)off * ld, ld, (int)o.op, b.L, b.Rt, ld, stm), "residual");
      // Intermediate sums are kept to 1e-12 of their size (F - A X_1 is
      // already far below F); the last one only to the accuracy the float32
      // correction solve can use.
      // The last sum feeds a float32 solve, so its core may be diagonalised
      // in float32 too.
      s = qr_round(h, b, b.L, b.Rt, ld, m, q, nullptr, last ? 1e-8 : 1e-12, KMAX, b.FU, b.FV, b.rs, ld,
                   last ? 2 : 1, last, &Kres, &rs0);
      if (s != LR_OK) return s;
      launches += 1 + kQrRoundLaunches;
      FUp = b.FU;
      FVp = b.FV;
      fr = Kres;
      fld = ld;
      off += c;
    }
    if (stuck) { worst = LR_ENOCONV; fail(h, worst, "residual rank too large for refinement (> 64)"); break; }
    if (Kres == 0) break;  // X solves the float64 system exactly
    double* Yl = b.FU;
    double* Yr = b.FV;
    // Correction D, written after X's R1 columns (room KMAX - R1).
    lr_mat res = {m, m, Kres, Kres, ld, Yl, nullptr, Yr};
    lr_mat D = {m, m, 0, KMAX - R1, ld, X.U + (size_t)R1 * ld, X.s + R1, X.V + (size_t)R1 * ld};
    // The correction is needed to a few digits only (a round cannot gain more
    // than the float32 solve resolves under the residual's cancellation), and
    // a looser tolerance keeps its rank well inside the 64-step cap.
    lr_options oc = o1;
    oc.eps = std::max(o1.eps, 1e-5);
    s = solve2d<float>(h, &res, &D, oc, plan);
    if (s != LR_OK && s != LR_ENOCONV) return s;  // ENOCONV: D cut to the room left, or cross cap
    launches += h->info.launches;
    const double sd = h->h_state->sigma0 * rs0;
    // Keep the correction's columns down to a tail below eps / 20 of X: the
    // rounding of X + D at eps drops them anyway, and a narrower core is
    // cheaper to diagonalise.
    int R2 = D.r;
    LR_CUDA(h, cudaMemcpyAsync(h->h_w, X.s, sizeof(double) * (R1 + R2), cudaMemcpyDeviceToHost, stm), "weights");
    LR_CUDA(h, cudaStreamSynchronize(stm), "weights");
    {
      double nx = 0.0, tail = 0.0;
      for (int j = 0; j < R1; ++j) nx += h->h_w[j] * h->h_w[j];
      const double lim = 0.05 * o.eps * std::sqrt(nx);
      while (R2 > 0) {
        const double v = h->h_w[R1 + R2 - 1] * rs0;
        if (std::sqrt(tail + v * v) > lim) break;
        tail += v * v;
        --R2;
      }
    }
    LR_CUDA(h, launch_scale_weights(R2, X.s + R1, b.rs, stm), "scale");
    // X + D = [XU, DU] diag(Xs, Ds) [XV, DV]^T, rounded at eps.  D lies
    // mostly in X's column space, which a Gram-based rounding would resolve
    // only to sqrt(eps64); the QR rounding keeps the factors orthonormal.
    int Rn = 0;
    double sig_new = 0.0;
    s = qr_round(h, b, X.U, X.V, ld, m, R1 + R2, X.s, o.eps, KMAX, X.U, X.V, X.s, ld, 0, false, &Rn, &sig_new);
    if (s != LR_OK && s != LR_ENOCONV) return s;
    if (s != LR_OK) worst = s;
    launches += 1 + kQrRoundLaunches;
    X.r = Rn;
    corr = sigX > 0.0 ? sd / sigX : 0.0;
    sigX = sig_new;
    ++done;
    // The error left after this round is about the correction times the
    // relative accuracy of the correction, estimated by the ratio of
    // successive corrections (0.05 before there is one: a float32 solve of
    // the residual loses accuracy to cancellation as the grid grows).
    const double rate = prev > 0.0 ? std::min(1.0, corr / prev) : 0.05;
    if (corr * rate <= 0.5 * o.eps) break;
    if (prev > 0.0 && corr > 0.5 * prev) break;  // no longer converging
    prev = corr;
  }
  // Copy the result into the caller's buffers.
  int R = X.r;
  if (R > sol->rmax) { R = sol->rmax; worst = LR_ENOCONV; fail(h, worst, "solution rank exceeds sol->rmax"); }
  const size_t col = sizeof(double) * (size_t)ld;
  if (R > 0) {
    LR_CUDA(h, cudaMemcpy2DAsync(sol->U, sizeof(double) * sol->ld, X.U, col, sizeof(double) * m, R,
                                 cudaMemcpyDeviceToDevice, stm), "copy U");
    LR_CUDA(h, cudaMemcpy2DAsync(sol->V, sizeof(double) * sol->ld, X.V, col, sizeof(double) * m, R,
                                 cudaMemcpyDeviceToDevice, stm), "copy V");
    LR_CUDA(h, cudaMemcpyAsync(sol->s, X.s, sizeof(double) * R, cudaMemcpyDeviceToDevice, stm), "copy s");
  }
  LR_CUDA(h, cudaStreamSynchronize(stm), "refined solve");
  sol->r = R;
  SolveState fin = first;
  fin.rank = R;
  fin.sigma0 = sigX;
  fin.cut = worst == LR_ENOCONV && first.converged;
  *h->h_state = fin;
  std::memcpy(h->h_piv, piv, sizeof piv);
  h->info.cluster_size = cs_first;
  h->last_cs = cs_first;
  h->info.launches = launches;
  h->info.refine_rounds = done;
  h->info.refine_corr = corr;
  return worst;
}

// Full-grid solve X = S ((S F S) / Lambda) S (Eq. flr:diag) with column
// transforms and transposes:
//   W1 = S F;  W2 = W1^T;  W1 = S W2 = (S F S)^T;
//   W2 = S (W1 / Lambda) = S Xh^T  (division fused into the transform input;
//                                   Lambda is symmetric);
//   W1 = W2^T = Xh S;  X = S W1.
template <typename T>
lr_status solve2d_full(lr_handle h, int m, const double* F, int ldf, double* X, int ldx, const lr_options& o,
                       Plan* plan) {
  const int ldw = round_up(m, 32);
  const size_t M = (size_t)1 << plan->logM;
  const size_t wbytes = align256(sizeof(T) * (size_t)ldw * m);
  const size_t sbytes = M > (size_t)kSmallM ? align256(sizeof(cpx<T>) * M * (size_t)m) : 256;
  const size_t need = 2 * wbytes + sbytes;
  if (need > h->ws3_bytes) {
    const lr_status sg = grow_ws(h, &h->ws3, &h->ws3_bytes, need, "full-grid workspace");
    if (sg != LR_OK) return sg;
  }
  char* base = static_cast<char*>(h->ws3);
  T* W1 = reinterpret_cast<T*>(base);
  T* W2 = reinterpret_cast<T*>(base + wbytes);
  void* scratch = base + 2 * wbytes;
  cudaStream_t stm = h->stream;
  const bool f32 = sizeof(T) == 4;
  auto cols = [&](const void* in, int ldi, void* out, int ldo) {
    ColumnSet cs;
    cs.in[0] = in; cs.ld_in[0] = ldi; cs.out[0] = out; cs.ld_out[0] = ldo; cs.ncol[0] = m;
    return cs;
  };
  ColumnSet c1 = cols(F, ldf, W1, ldw);
  LR_CUDA(h, launch_dst<T>(*plan, c1, IoType::F64, IoType::WORK, scratch, h->num_sms, stm), "full: S F");
  LR_CUDA(h, launch_transpose<T>(W1, ldw, m, m, W2, ldw, stm), "full: transpose");
  ColumnSet c2 = cols(W2, ldw, W1, ldw);
  LR_CUDA(h, launch_dst<T>(*plan, c2, IoType::WORK, IoType::WORK, scratch, h->num_sms, stm), "full: S F S");
  ColumnSet c3 = cols(W1, ldw, W2, ldw);
  c3.sym_a = f32 ? (const void*)plan->sym_a32[o.op] : (const void*)plan->sym_a64[o.op];
  c3.sym_b = f32 ? (const void*)plan->sym_b32[o.op] : (const void*)plan->sym_b64[o.op];
  LR_CUDA(h, launch_dst<T>(*plan, c3, IoType::DIV, IoType::WORK, scratch, h->num_sms, stm), "full: S Xh^T");
  LR_CUDA(h, launch_transpose<T>(W2, ldw, m, m, W1, ldw, stm), "full: transpose");
  ColumnSet c4 = cols(W1, ldw, X, ldx);
  LR_CUDA(h, launch_dst<T>(*plan, c4, IoType::WORK, IoType::F64, scratch, h->num_sms, stm), "full: S Xh S");
  LR_CUDA(h, cudaStreamSynchronize(stm), "full-grid solve");
  return LR_OK;
}

// Exponential-sum solve of the 5-point problem (Section 4.1, the "known
// approaches" the cross is compared with): with 1/lambda ~ sum_q w_q
// exp(-t_q lambda) (sinc quadrature of int exp(s - lambda e^s) ds) and
// Lambda_ij = mu_i + mu_j,
//   Xh ~ sum_q w_q (E_q Uh) (E_q Vh)^T,  E_q = diag(exp(-t_q mu)),
// accumulated in chunks of terms (each rounding sees at most 64 columns) by
// float64 QR rounding; float64 transforms.
lr_status solve2d_expsum(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options& o, Plan* plan,
                         int* nterms) {
  const int m = rhs->n1, r = rhs->r;
  const int ld = m + (m & 1);
  RefineBufs b;
  Carve sizing;
  carve_refine(sizing, b, ld, m);
  if (sizing.off > h->ws2_bytes) {
    const lr_status sg = grow_ws(h, &h->ws2, &h->ws2_bytes, sizing.off, "exp-sum buffers");
    if (sg != LR_OK) return sg;
  }
  Carve cv;
  cv.base = static_cast<char*>(h->ws2);
  carve_refine(cv, b, ld, m);
  cudaStream_t stm = h->stream;
  // Quadrature over the spectrum [2 mu_1, 2 mu_m] at eps / 10 (nodes on the
  // host: step, ends and weights as stated for the sinc rule).
  const double N = m + 1.0;
  const double mu1 = 4.0 * N * N * std::pow(std::sin(M_PI / (2.0 * N)), 2);
  const double mum = 4.0 * N * N * std::pow(std::cos(M_PI / (2.0 * N)), 2);
  const double lo = 2.0 * mu1, hi = 2.0 * mum, eq = o.eps / 10.0;
  const double tau = M_PI * M_PI / (std::log(1.0 / eq) + std::log(32.0));
  const double s_min = std::log(eq / (4.0 * hi));
  const double s_max = std::log((std::log(hi / eq) + 2.0) / lo);
  const int Q = (int)std::ceil((s_max - s_min) / tau) + 1;
  if (Q > 2 * KMAX) return fail(h, LR_EINVAL, "exp-sum: too many quadrature terms (eps too small)");
  std::vector<double> tw(2 * Q);
  for (int k = 0; k < Q; ++k) {
    tw[k] = std::exp(s_min + k * tau);
    tw[Q + k] = tau * tw[k];
  }
  // forward transforms of the factors (float64) into FU, FV
  const size_t M = (size_t)1 << plan->logM;
  // four-step scratch for the larger of the two transforms (2r and 2R <= 2 KMAX columns)
  lr_status s = ensure_ws(h, M > (size_t)kSmallM ? M * 2 * (size_t)KMAX * sizeof(cpx<double>) + 256 : 256);
  if (s != LR_OK) return s;
  {
    ColumnSet cs;
    cs.in[0] = rhs->U; cs.in[1] = rhs->V;
    cs.ld_in[0] = rhs->ld; cs.ld_in[1] = rhs->ld;
    cs.out[0] = b.FU; cs.out[1] = b.FV;
    cs.ld_out[0] = ld; cs.ld_out[1] = ld;
    cs.ncol[0] = r; cs.ncol[1] = r;
    LR_CUDA(h, launch_dst<double>(*plan, cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm), "exp-sum: forward");
  }
  double* dt = nullptr;
  double* dw = nullptr;
  if (Q <= 2 * KMAX) {  // nodes and weights in b.aux (4 KMAX values)
    dt = b.aux;
    dw = b.aux + 2 * KMAX;
    LR_CUDA(h, cudaMemcpyAsync(dt, tw.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, stm), "nodes");
    LR_CUDA(h, cudaMemcpyAsync(dw, tw.data() + Q, sizeof(double) * Q, cudaMemcpyHostToDevice, stm), "weights");
  }
  const double* mu = plan->sym_a64[LR_OP_5PT];
  int K = 0;
  double sig = 0.0;
  for (int k = 0; k < Q;) {
    const int c = std::min(Q - k, (KMAX - K) / r);
    if (c < 1) return fail(h, LR_ENOCONV, "exp-sum: running rank leaves no room for a term");
    if (K > 0) {
      LR_CUDA(h, cudaMemcpyAsync(b.L, b.XU, sizeof(double) * (size_t)ld * K, cudaMemcpyDeviceToDevice, stm), "stack");
      LR_CUDA(h, cudaMemcpyAsync(b.Rt, b.XV, sizeof(double) * (size_t)ld * K, cudaMemcpyDeviceToDevice, stm), "stack");
    }
    LR_CUDA(h, launch_scale_copy(K, b.Xs, 1.0, b.rs, stm), "weights");
    LR_CUDA(h, launch_scale_copy(c * r, nullptr, 1.0, b.rs + K, stm), "weights");
    LR_CUDA(h, launch_expsum_cols(m, r, c, b.FU, b.FV, ld, mu, dt + k, dw + k, b.L, b.Rt, ld, K, stm), "terms");
    const bool last = k + c == Q;
    s = qr_round(h, b, b.L, b.Rt, ld, m, K + c * r, b.rs, last ? o.eps : o.eps / 4.0, KMAX, b.XU, b.XV, b.Xs, ld,
                 0, false, &K, &sig);
    if (s != LR_OK && s != LR_ENOCONV) return s;
    k += c;
  }
  // inverse transforms into the caller's factors
  const int R = std::min(K, sol->rmax);
  if (R > 0) {
    ColumnSet cs;
    cs.in[0] = b.XU; cs.in[1] = b.XV;
    cs.ld_in[0] = ld; cs.ld_in[1] = ld;
    cs.out[0] = sol->U; cs.out[1] = sol->V;
    cs.ld_out[0] = sol->ld; cs.ld_out[1] = sol->ld;
    cs.ncol[0] = R; cs.ncol[1] = R;
    LR_CUDA(h, launch_dst<double>(*plan, cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm), "exp-sum: inverse");
    LR_CUDA(h, cudaMemcpyAsync(sol->s, b.Xs, sizeof(double) * R, cudaMemcpyDeviceToDevice, stm), "copy s");
  }
  LR_CUDA(h, cudaStreamSynchronize(stm), "exp-sum solve");
  sol->r = R;
  if (nterms) *nterms = Q;
  if (R < K) return fail(h, LR_ENOCONV, "solution rank exceeds sol->rmax; result truncated");
  return LR_OK;
}

constexpr int kBatchStreams = 32;

lr_status ensure_batch_streams(lr_handle h) {
  if (h->bstreams[0]) return LR_OK;
  for (int i = 0; i < kBatchStreams; ++i) {
    LR_CUDA(h, cudaStreamCreateWithFlags(&h->bstreams[i], cudaStreamNonBlocking), "stream create");
    LR_CUDA(h, cudaEventCreateWithFlags(&h->bjoin[i], cudaEventDisableTiming), "event create");
  }
  LR_CUDA(h, cudaEventCreateWithFlags(&h->bfork, cudaEventDisableTiming), "event create");
  return LR_OK;
}

// Per-problem ranks and statuses of a finished batched call, from the pinned
// status record its stream wrote last.
lr_status collect_batch(lr_handle h, int batch, lr_mat* sol, lr_status* per_problem) {
  lr_status worst = LR_OK;
  for (int i = 0; i < batch; ++i) {
    const SolveState& hs = h->h_bstate[i];
    sol[i].r = hs.rank;
    const lr_status si = hs.status ? static_cast<lr_status>(hs.status)
                                   : ((!hs.converged || hs.cut) ? LR_ENOCONV : LR_OK);
    if (per_problem) per_problem[i] = si;
    if (si != LR_OK && worst != LR_ENONFINITE) worst = si;
  }
  if (worst != LR_OK) fail(h, worst, "some problems did not converge or were cut (see per_problem)");
  return worst;
}

template <typename T>
lr_status solve2d_batched_streams(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options& o,
                                  const std::vector<Plan*>& plans, lr_status* per_problem) {
  std::vector<SolveGeom> geo(batch);
  std::vector<size_t> off(batch);
  Carve c;
  for (int i = 0; i < batch; ++i) {
    geo[i] = geom_of(rhs[i].n1, rhs[i].r, sol[i].rmax, o, *plans[i]);
    off[i] = c.off;
    carve_slice<T>(c, geo[i]);
  }
  const size_t st_off = c.off;
  c.take<SolveState>(sizeof(SolveState) * batch);
  lr_status s = ensure_ws(h, c.off);
  if (s != LR_OK) return s;
  if ((s = ensure_batch_streams(h)) != LR_OK) return s;
  if (h->bstate_cap < batch) {
    if (h->h_bstate) cudaFreeHost(h->h_bstate);
    h->h_bstate = nullptr;
    h->bstate_cap = 0;
    if (cudaMallocHost(&h->h_bstate, sizeof(SolveState) * batch) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, LR_ENOMEM, "pinned status buffer");
    }
    h->bstate_cap = batch;
    ++h->ws_gen;  // graphs captured with the old buffer are stale
  }
  char* base = static_cast<char*>(h->ws);
  SolveState* states = reinterpret_cast<SolveState*>(base + st_off);
  // Longest-processing-time order, dealt round-robin over the streams.
  std::vector<int> order(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)geo[a].m * (geo[a].r + 16) > (double)geo[b].m * (geo[b].r + 16);
  });
  int launches = 0;
  for (int i = 0; i < batch; ++i) launches += launches_of(geo[i]);
  // Throughput mode: unless the caller fixed it, give each cross about 2048
  // indices per CTA (or the autotuned number).  Its per-step cost is mostly a
  // fixed latency, so fewer, fuller CTAs per problem spend less SM time and
  // let more problems run at once (a single solve uses about 1024 indices per
  // CTA for latency).
  std::vector<lr_options> popt(batch, o);
  const int ipc = h->batch_ipc[sizeof(T) == 4 ? 1 : 0];
  if (o.cluster_size == 0)
    for (int i = 0; i < batch; ++i) {
      int cs = (geo[i].m + ipc - 1) / ipc;
      popt[i].cluster_size = cs < 1 ? 1 : (cs > 16 ? 16 : cs);
    }
  const bool graph = (o.flags & LR_FLAG_GRAPH) != 0;
  s = run_maybe_graph(h, graph, key_of("batch", rhs, batch, sol, o), [&](cudaStream_t main) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaEventRecord(h->bfork, main)) != cudaSuccess) return e;
    for (int j = 0; j < kBatchStreams; ++j)
      if ((e = cudaStreamWaitEvent(h->bstreams[j], h->bfork, 0)) != cudaSuccess) return e;
    for (int n = 0; n < batch; ++n) {
      const int i = order[n];
      Carve ci;
      ci.base = base + off[i];
      const Slice<T> w = carve_slice<T>(ci, geo[i]);
      int used = 0;
      if ((e = enqueue_solve<T>(h, &rhs[i], &sol[i], popt[i], *plans[i], geo[i], w, &states[i],
                                h->bstreams[n % kBatchStreams], nullptr, &used)) != cudaSuccess)
        return e;
    }
    for (int j = 0; j < kBatchStreams; ++j) {
      if ((e = cudaEventRecord(h->bjoin[j], h->bstreams[j])) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(main, h->bjoin[j], 0)) != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(h->h_bstate, states, sizeof(SolveState) * batch, cudaMemcpyDeviceToHost, main);
  });
  if (s != LR_OK) return s;
  h->info.launches = launches;
  if (o.flags & LR_FLAG_ASYNC) return LR_OK;
  LR_CUDA(h, cudaStreamSynchronize(h->stream), "batched solve");
  return collect_batch(h, batch, sol, per_problem);
}

// Twiddles exp(-2 pi i q / 4096) of the batched transforms, per precision.
lr_status ensure_tw4096(lr_handle h, bool f32) {
  void*& t = h->tw4096[f32 ? 1 : 0];
  if (t) return LR_OK;
  std::vector<double> re(4096), im(4096);
  for (int q = 0; q < 4096; ++q) {
    // angle reduced to the first octant in integers (as the plan tables)
    const int p = q / 1024, r = q % 1024;
    double c, sn;
    if (2 * r <= 1024) { const double th = 2.0 * M_PI * r / 4096.0; c = std::cos(th); sn = std::sin(th); }
    else { const double th = 2.0 * M_PI * (1024 - r) / 4096.0; c = std::sin(th); sn = std::cos(th); }
    double x, y;  // exp(+2 pi i q / 4096)
    switch (p) { case 0: x = c; y = sn; break; case 1: x = -sn; y = c; break;
                 case 2: x = -c; y = -sn; break; default: x = sn; y = -c; }
    re[q] = x;
    im[q] = -y;   // conjugate: exp(-2 pi i q / 4096)
  }
  const size_t w = f32 ? sizeof(float) : sizeof(double);
  std::vector<char> buf(4096 * 2 * w);
  for (int q = 0; q < 4096; ++q) {
    if (f32) { float* f = reinterpret_cast<float*>(buf.data()); f[2 * q] = (float)re[q]; f[2 * q + 1] = (float)im[q]; }
    else { double* d = reinterpret_cast<double*>(buf.data()); d[2 * q] = re[q]; d[2 * q + 1] = im[q]; }
  }
  if (cudaMalloc(&t, buf.size()) != cudaSuccess) {
    cudaGetLastError();
    t = nullptr;
    return fail(h, LR_ENOMEM, "twiddle table");
  }
  LR_CUDA(h, cudaMemcpy(t, buf.data(), buf.size(), cudaMemcpyHostToDevice), "twiddle table");
  return LR_OK;
}

// Host-built description of a phase-batched solve: the problem records and
// the item lists of every launch, in one block uploaded to the device.
struct BatchLayout {
  std::vector<char> blob;  // [BatchProb x n][int lists]
  size_t probs_off = 0;
  struct ListRef { size_t list, start; int n, items, slog, fused_logh; };
  ListRef fwd_small{}, fwd_col{}, fwd_row{}, inv_small{}, inv_col{}, inv_row{}, rot{};
  struct CrossGroup { size_t list; int n, cs, rows; };
  std::vector<CrossGroup> cross;
  BatchItems items(const ListRef& r, const char* dev) const {
    BatchItems b;
    b.list = reinterpret_cast<const int*>(dev + r.list);
    b.start = reinterpret_cast<const int*>(dev + r.start);
    b.n = r.n;
    b.items = r.items;
    b.slog = r.slog;
    b.fused_logh = r.fused_logh;
    return b;
  }
};

// True if every problem fits the phase-batched kernels in this precision.
bool batch_phased_fits(int batch, const lr_mat* rhs, bool f32) {
  // transform length M <= 2^17 (the batched four-step twiddle tables)
  const int lim = std::min(65536, 16 * batch_cross_max_rows(f32));
  for (int i = 0; i < batch; ++i)
    if (rhs[i].n1 > lim) return false;
  return true;
}

template <typename T>
lr_status solve2d_batched_phased(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options& o,
                                 const std::vector<Plan*>& plans, lr_status* per_problem) {
  const bool f32 = sizeof(T) == 4;
  lr_status s;
  if ((s = ensure_tw4096(h, f32)) != LR_OK) return s;
  // ---- workspace: per problem the single-solve slice plus the rotated
  // skeleton W (m x 2 ncap), then the solve states
  std::vector<SolveGeom> geo(batch);
  std::vector<size_t> off(batch), woff(batch);
  Carve c;
  for (int i = 0; i < batch; ++i) {
    geo[i] = geom_of(rhs[i].n1, rhs[i].r, sol[i].rmax, o, *plans[i]);
    off[i] = c.off;
    carve_slice<T>(c, geo[i]);
    woff[i] = c.off;
    c.take<char>(sizeof(T) * (size_t)geo[i].ldw * 2 * geo[i].ncap_out);
  }
  const size_t st_off = c.off;
  c.take<SolveState>(sizeof(SolveState) * batch);
  const size_t live_off = c.off;  // device-written item tables of the inverse transforms
  c.take<int>(sizeof(int) * 3 * ((size_t)batch + 1));
  if ((s = ensure_ws(h, c.off)) != LR_OK) return s;
  if (h->bstate_cap < batch) {
    if (h->h_bstate) cudaFreeHost(h->h_bstate);
    h->h_bstate = nullptr;
    h->bstate_cap = 0;
    if (cudaMallocHost(&h->h_bstate, sizeof(SolveState) * batch) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, LR_ENOMEM, "pinned status buffer");
    }
    h->bstate_cap = batch;
    ++h->ws_gen;
  }
  if ((s = ensure_batch_streams(h)) != LR_OK) return s;
  int* live_tab = reinterpret_cast<int*>(static_cast<char*>(h->ws) + live_off);
  char* base = static_cast<char*>(h->ws);
  SolveState* states = reinterpret_cast<SolveState*>(base + st_off);
  // ---- problem records
  BatchLayout L;
  std::vector<BatchProb> P(batch);
  const int pi = f32 ? 1 : 0;
  for (int i = 0; i < batch; ++i) {
    const SolveGeom& g = geo[i];
    const Plan& pl = *plans[i];
    Carve ci;
    ci.base = base + off[i];
    const Slice<T> w = carve_slice<T>(ci, g);
    BatchProb& b = P[i];
    b.m = g.m; b.r = g.r; b.kcap = g.kcap; b.ldw = g.ldw; b.ncap = g.ncap_out;
    b.logM = pl.logM; b.logM1 = pl.logM1; b.logM2 = pl.logM2;
    b.ld_in = rhs[i].ld; b.ld_out = sol[i].ld;
    b.U = rhs[i].U; b.V = rhs[i].V;
    b.Uo = sol[i].U; b.Vo = sol[i].V; b.so = sol[i].s;
    b.Uh = w.Uh; b.Vh = w.Vh; b.C = w.C; b.R = w.R; b.Tc = w.Tc; b.Tr = w.Tr;
    b.W = base + woff[i];
    b.work = w.work;
    b.GC = w.GC; b.GR = w.GR; b.d = w.d; b.I = w.I; b.J = w.J;
    b.st = &states[i];
    const TablesT& tb = f32 ? pl.t32 : pl.t64;
    b.chirp = tb.chirp; b.tw = tb.tw; b.bhat = tb.bhat; b.bres = tb.bhat_rs;
    b.sa = f32 ? (const void*)pl.sym_a32[o.op] : (const void*)pl.sym_a64[o.op];
    b.sb = f32 ? (const void*)pl.sym_b32[o.op] : (const void*)pl.sym_b64[o.op];
  }
  // ---- item lists.  Cost order (longest first) for every list.
  std::vector<int> order(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)geo[a].m * (geo[a].r + 16) > (double)geo[b].m * (geo[b].r + 16);
  });
  std::vector<int> ints;
  auto add_list = [&](std::vector<int> lst, std::vector<int> cnt, BatchLayout::ListRef& ref) {
    ref.n = (int)lst.size();
    ref.list = ints.size() * sizeof(int);
    ints.insert(ints.end(), lst.begin(), lst.end());
    ref.start = ints.size() * sizeof(int);
    int acc = 0;
    for (int c2 : cnt) { ints.push_back(acc); acc += c2; }
    ints.push_back(acc);
    ref.items = acc;
  };
  // the one-pass transform runs one CTA per column: only batches with enough
  // columns to fill the GPU take it
  int fwd_cols = 0;
  for (int i = 0; i < batch; ++i) fwd_cols += 2 * geo[i].r;
  const int fused_lh =
      f32 && h->dst_fused[pi] && fwd_cols >= h->num_sms / 2 ? kFusedLogH32 : 0;
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int> ls, cs_, lf, cf, rf;
    int slog_s = 0, slog_c = 0, slog_r = 0;  // largest FFT stage each launch needs
    for (int i : order) {
      const int ncols = dir == 0 ? 2 * geo[i].r : 2 * geo[i].ncap_out;
      const int logM = plans[i]->logM;
      if (logM <= 12) {
        const int nf = 1 << (12 - logM);
        ls.push_back(i);
        cs_.push_back((ncols + nf - 1) / nf);
        slog_s = std::max(slog_s, logM - 2);
      } else if (fused_lh && logM >= fused_lh - 1) {  // one pass per column (an item:
                                                      // 2^(LH - min(logM, LH)) columns)
        const int nf = 1 << (fused_lh - std::min(logM, fused_lh));
        lf.push_back(i);
        cf.push_back((ncols + nf - 1) / nf);
      } else {
        const int logM1 = plans[i]->logM1, logM2 = plans[i]->logM2;
        lf.push_back(i);
        cf.push_back(ncols * ((1 << logM1) >> (12 - logM2)));
        rf.push_back(ncols * ((1 << logM2) >> (12 - logM1)));
        slog_c = std::max(slog_c, logM2 - 2);
        slog_r = std::max(slog_r, logM1 - 2);
      }
    }
    BatchLayout::ListRef& rs_ = dir == 0 ? L.fwd_small : L.inv_small;
    BatchLayout::ListRef& rc_ = dir == 0 ? L.fwd_col : L.inv_col;
    BatchLayout::ListRef& rr_ = dir == 0 ? L.fwd_row : L.inv_row;
    add_list(ls, cs_, rs_);
    add_list(lf, cf, rc_);
    if (fused_lh) add_list({}, {}, rr_);
    else add_list(lf, rf, rr_);
    rc_.fused_logh = fused_lh;
    rs_.slog = slog_s;
    rc_.slog = slog_c;
    rr_.slog = slog_r;
    // the row-pass list shares problems with the column-pass list
  }
  {
    std::vector<int> lr_, cr;
    for (int i : order) { lr_.push_back(i); cr.push_back((geo[i].m + 255) / 256); }
    add_list(lr_, cr, L.rot);
  }
  // cross groups: cluster sizes 1, 2, 4, 8, 16 so that each CTA has at most
  // rows_per_cta indices (more only at 16 CTAs)
  const int rows = std::min(h->cross_rows[pi], batch_cross_max_rows(f32));
  for (int cs : {16, 8, 4, 2, 1}) {
    std::vector<int> lst;
    int mx = 0;
    for (int i : order) {
      const int m = geo[i].m;
      int need = 1;
      while (need < 16 && (long long)need * rows < m) need *= 2;
      if (o.cluster_size > 0) {  // the caller's cluster size (a power of two), enough for the rows
        int want = 1;
        while (want < o.cluster_size && want < 16) want *= 2;
        need = std::max(want, need);
        while (need > 1 && (long long)(need / 2) * batch_cross_max_rows(f32) >= m && need > want) need /= 2;
      }
      if (need == cs) { lst.push_back(i); mx = std::max(mx, (m + cs - 1) / cs); }
    }
    if (lst.empty()) continue;
    BatchLayout::CrossGroup g;
    g.list = ints.size() * sizeof(int);
    g.n = (int)lst.size();
    g.cs = cs;
    g.rows = mx;
    ints.insert(ints.end(), lst.begin(), lst.end());
    L.cross.push_back(g);
  }
  const size_t pbytes = align256(sizeof(BatchProb) * batch);
  L.blob.assign(pbytes + ints.size() * sizeof(int), 0);
  std::memcpy(L.blob.data(), P.data(), sizeof(BatchProb) * batch);
  std::memcpy(L.blob.data() + pbytes, ints.data(), ints.size() * sizeof(int));
  auto shift = [&](BatchLayout::ListRef& r) { r.list += pbytes; r.start += pbytes; };
  shift(L.fwd_small); shift(L.fwd_col); shift(L.fwd_row);
  shift(L.inv_small); shift(L.inv_col); shift(L.inv_row); shift(L.rot);
  for (auto& g : L.cross) g.list += pbytes;
  // ---- the enqueued steps, given the device copy of the block
  BatchCrossParams cp;
  cp.tol = o.aca_tol_factor * o.eps;
  cp.probes = o.probes;
  cp.seed = o.seed;
  cp.max_probe_rounds = 4;
  cp.max_zero_rows = 16;
  const int nsm = h->num_sms;
  const void* tw = h->tw4096[pi];
  const int col_launches = fused_lh ? 1 : 3;
  const int launches = (L.fwd_small.items > 0) + col_launches * (L.fwd_col.items > 0) + (int)L.cross.size() + 3 +
                       (L.inv_small.items > 0) + col_launches * (L.inv_col.items > 0);
  const bool timing = (o.flags & LR_FLAG_TIMING) != 0;
  if (timing && (s = ensure_events(h)) != LR_OK) return s;
  auto mark = [&](int i, cudaStream_t stm) -> cudaError_t {
    return timing ? cudaEventRecord(h->ev[i], stm) : cudaSuccess;
  };
  auto body = [&](cudaStream_t main, const char* dev) -> cudaError_t {
    cudaError_t e;
    const BatchProb* dp = reinterpret_cast<const BatchProb*>(dev);
    if ((e = cudaMemsetAsync(states, 0, sizeof(SolveState) * batch, main)) != cudaSuccess) return e;
    if ((e = mark(0, main)) != cudaSuccess) return e;
    {
      NvtxRange r("lr:forward_dst");
      if ((e = launch_batch_dst<T>(dp, 0, L.items(L.fwd_small, dev), L.items(L.fwd_col, dev),
                                   L.items(L.fwd_row, dev), tw, nsm, main)) != cudaSuccess)
        return e;
      if ((e = mark(1, main)) != cudaSuccess) return e;
    }
    {
      NvtxRange r("lr:cross");
      // the cluster-size groups run concurrently on forked streams
      const int ng = (int)L.cross.size();
      if (ng > 1) {
        if ((e = cudaEventRecord(h->bfork, main)) != cudaSuccess) return e;
        for (int j = 0; j < ng; ++j)
          if ((e = cudaStreamWaitEvent(h->bstreams[j], h->bfork, 0)) != cudaSuccess) return e;
      }
      for (int j = 0; j < ng; ++j) {
        const auto& g = L.cross[j];
        cudaStream_t sj = ng > 1 ? h->bstreams[j] : main;
        if ((e = launch_batch_cross<T>(dp, reinterpret_cast<const int*>(dev + g.list), g.n, g.cs, g.rows, cp,
                                       sj)) != cudaSuccess)
          return e;
      }
      if (ng > 1)
        for (int j = 0; j < ng; ++j) {
          if ((e = cudaEventRecord(h->bjoin[j], h->bstreams[j])) != cudaSuccess) return e;
          if ((e = cudaStreamWaitEvent(main, h->bjoin[j], 0)) != cudaSuccess) return e;
        }
      if ((e = mark(2, main)) != cudaSuccess) return e;
    }
    {
      NvtxRange r("lr:rounding");
      if ((e = launch_batch_core<T>(dp, batch, o.eps, f32, main)) != cudaSuccess) return e;
      if ((e = launch_batch_rotate<T>(dp, L.items(L.rot, dev), nsm, main)) != cudaSuccess) return e;
      if ((e = mark(3, main)) != cudaSuccess) return e;
    }
    {
      NvtxRange r("lr:inverse_dst");
      // only the kept columns (2 R per problem) are transformed: their item
      // tables are counted on the device once the ranks are known
      BatchItems ism = L.items(L.inv_small, dev), icol = L.items(L.inv_col, dev), irow = L.items(L.inv_row, dev);
      ism.start = live_tab;
      icol.start = live_tab + (batch + 1);
      irow.start = live_tab + 2 * (batch + 1);
      ism.live = icol.live = irow.live = 1;
      if ((e = launch_batch_live_items(dp, ism, icol, irow, main)) != cudaSuccess) return e;
      if ((e = launch_batch_dst<T>(dp, 1, ism, icol, irow, tw, nsm, main)) != cudaSuccess) return e;
      if ((e = mark(4, main)) != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(h->h_bstate, states, sizeof(SolveState) * batch, cudaMemcpyDeviceToHost, main);
  };
  const bool graph = (o.flags & LR_FLAG_GRAPH) != 0 && !timing;
  h->timed = timing;
  if (graph) {
    // the graph bakes in the device copy of the block: one copy per graph
    const std::string key = key_of("phased", rhs, batch, sol, o) + "|ipc" + std::to_string(rows) + "|ws" +
                            std::to_string(h->ws_gen);
    auto it = h->graph_desc.find(key);
    char* dev = it != h->graph_desc.end() ? it->second : nullptr;
    if (!dev) {
      if (h->graphs.size() >= 32) {  // make room before allocating (bounded cache)
        cudaStreamSynchronize(h->stream);
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
        for (auto& kv : h->graph_desc) cudaFree(kv.second);
        h->graph_desc.clear();
      }
      if (cudaMalloc(&dev, L.blob.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LR_ENOMEM, "batch descriptor block");
      }
      cudaError_t e = cudaMemcpy(dev, L.blob.data(), L.blob.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) { cudaFree(dev); return cuda_fail(h, e, "batch descriptor upload"); }
      h->graph_desc[key] = dev;
    }
    s = run_maybe_graph(h, true, key, [&](cudaStream_t stm) { return body(stm, dev); });
  } else {
    // stream-ordered upload through a pinned staging buffer
    if (L.blob.size() > h->bdesc_cap) {
      if (h->bdesc) { cudaStreamSynchronize(h->stream); cudaFree(h->bdesc); }
      h->bdesc = nullptr;
      h->bdesc_cap = 0;
      if (cudaMalloc(&h->bdesc, L.blob.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LR_ENOMEM, "batch descriptor block");
      }
      h->bdesc_cap = L.blob.size();
    }
    if (!h->bdesc_ev) LR_CUDA(h, cudaEventCreateWithFlags(&h->bdesc_ev, cudaEventDisableTiming), "event create");
    LR_CUDA(h, cudaEventSynchronize(h->bdesc_ev), "staging buffer");
    if (L.blob.size() > h->h_bdesc_cap) {
      if (h->h_bdesc) cudaFreeHost(h->h_bdesc);
      h->h_bdesc = nullptr;
      h->h_bdesc_cap = 0;
      if (cudaMallocHost(&h->h_bdesc, L.blob.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LR_ENOMEM, "pinned descriptor buffer");
      }
      h->h_bdesc_cap = L.blob.size();
    }
    std::memcpy(h->h_bdesc, L.blob.data(), L.blob.size());
    LR_CUDA(h, cudaMemcpyAsync(h->bdesc, h->h_bdesc, L.blob.size(), cudaMemcpyHostToDevice, h->stream), "upload");
    LR_CUDA(h, cudaEventRecord(h->bdesc_ev, h->stream), "event record");
    cudaError_t e = body(h->stream, h->bdesc);
    s = e == cudaSuccess ? LR_OK : cuda_fail(h, e, "enqueue");
  }
  if (s != LR_OK) return s;
  h->info.launches = launches;
  if (o.flags & LR_FLAG_ASYNC) return LR_OK;
  LR_CUDA(h, cudaStreamSynchronize(h->stream), "batched solve");
  return collect_batch(h, batch, sol, per_problem);
}

// Batched solves: the phase-batched kernels when every problem fits them
// (and the caller did not ask for the per-problem stream form), else one
// launch chain per problem over the internal streams.
template <typename T>
lr_status solve2d_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options& o,
                          const std::vector<Plan*>& plans, lr_status* per_problem, bool phased_ok = true) {
  const bool f32 = sizeof(T) == 4;
  if (phased_ok && !(o.flags & LR_FLAG_BATCH_STREAMS) &&
      batch_phased_fits(batch, rhs, f32))
    return solve2d_batched_phased<T>(h, batch, rhs, sol, o, plans, per_problem);
  return solve2d_batched_streams<T>(h, batch, rhs, sol, o, plans, per_problem);
}

// ---------------------------------------------------------------------------
// Low-rank Uzawa solve of the 2D Stokes problem on semi-staggered grids
// (Section 2, Eq. flr:stprob and Eq. flr:schur; Section 5): conjugate
// gradients on (B^T A^-1 B) p = B^T A^-1 f with every iterate in low-rank
// format, every sum rounded in float64 at eps, the d = 2 velocity solves of a
// Schur product batched, the CG scalars in float64.
// ---------------------------------------------------------------------------
struct LrDev {
  double *U = nullptr, *s = nullptr, *V = nullptr;
  int r = 0;
};

struct StokesCtx {
  lr_handle h;
  int n, ldp, ldv;
  RefineBufs b;
  LrDev P, R, D, Q, T;               // pressure-sized (n x KMAX), T: scratch result
  LrDev G;                           // the divergence right-hand side g (rounded copy)
  bool has_g = false;
  double *RU[2], *RV[2];             // velocity right-hand sides ((n-1) x KMAX, weights folded)
  double *WU[2], *Ws[2], *WV[2];     // velocity solutions
  double *wts, *gm0, *gm1, *cs, *E;  // weights, cross Gram matrices, column sums, kernel modes
  double* xpart;                     // cross Gram partials (32-row blocks)
  double* hbuf;                      // pinned host: 2 KMAX^2 + 4 KMAX
  Plan* plan;
  lr_options oin;                    // inner solves
  double eps;
  int launches = 0;
  int escalations = 0;               // mixed velocity solves repeated in float64
  bool cut = false;                  // a low-rank sum needed more than 64 columns
  bool gmres = false;                // inexact GMRES instead of CG
  std::vector<LrDev> K;              // GMRES: Krylov basis (kGmresRestart + 1 vectors)
};

constexpr int kGmresRestart = 20;
// Loosest relative accuracy of a relaxed GMRES product: looser products lose
// the Krylov relation through the amplification of B^T.
constexpr double kGmresMaxDelta = 1e-4;

void carve_stokes(Carve& c, StokesCtx& x) {
  carve_refine(c, x.b, x.ldp, x.n);
  const size_t cp = sizeof(double) * (size_t)x.ldp * KMAX, cv = sizeof(double) * (size_t)x.ldv * KMAX;
  for (LrDev* d : {&x.P, &x.R, &x.D, &x.Q, &x.T, &x.G}) {
    d->U = c.take<double>(cp);
    d->V = c.take<double>(cp);
    d->s = c.take<double>(sizeof(double) * KMAX);
  }
  for (int k = 0; k < 2; ++k) {
    x.RU[k] = c.take<double>(cv);
    x.RV[k] = c.take<double>(cv);
    x.WU[k] = c.take<double>(cv);
    x.WV[k] = c.take<double>(cv);
    x.Ws[k] = c.take<double>(sizeof(double) * KMAX);
  }
  x.wts = c.take<double>(sizeof(double) * 2 * KMAX);
  x.gm0 = c.take<double>(sizeof(double) * KMAX * KMAX);
  x.gm1 = c.take<double>(sizeof(double) * KMAX * KMAX);
  x.cs = c.take<double>(sizeof(double) * 4 * KMAX);
  x.E = c.take<double>(sizeof(double) * 2 * x.ldp);
  x.xpart = c.take<double>(sizeof(double) * KMAX * KMAX * (size_t)((x.n + 31) / 32));
  x.K.assign(x.gmres ? kGmresRestart + 1 : 0, LrDev{});
  for (LrDev& d : x.K) {
    d.U = c.take<double>(cp);
    d.V = c.take<double>(cp);
    d.s = c.take<double>(sizeof(double) * KMAX);
  }
}

// A term U diag(coef s) V^T of a sum (s null: ones; U, V leading dim ld).
struct Term {
  const double* U;
  const double* s;
  const double* V;
  int r, ld;
  double coef;
};

// dst = round(sum of terms), rows x rows matrices, dst orthonormal with
// leading dimension ldo: relative tolerance eps, and abs_tol > 0 also allows
// an absolute dropped tail.  Up to 64 columns the sum is rounded at once; a
// wider one is accumulated in chunks, the running result plus as many further
// columns as fit in 64, each partial rounding at eps / 4 and abs_tol / 2.  An
// absolute truncation does not depend on how much the terms cancel (the CG
// update r - alpha q cancels to a fraction of both), so the result stays
// within max(eps ||sum||, abs_tol) of the exact sum, where dropping columns
// by weight before the rounding would not.  Columns enter in term order, each
// term's in descending weight.  dst must not alias a term; x.cut is set if
// the running rank leaves no room for the rest.
lr_status sum_round(StokesCtx& x, int rows, const std::vector<Term>& terms, LrDev& dst, int ldo,
                    double abs_tol = 0.0) {
  lr_handle h = x.h;
  cudaStream_t stm = h->stream;
  std::vector<Term> tv;
  int q = 0;
  for (const Term& t : terms)
    if (t.r > 0) {
      tv.push_back(t);
      q += t.r;
    }
  if (q == 0) { dst.r = 0; return LR_OK; }
  const bool single = q <= KMAX;
  size_t ti = 0;  // next column: term ti, column tj
  int tj = 0;
  int K = 0;      // rank of the running result (in dst)
  while (ti < tv.size()) {
    if (K >= KMAX) { x.cut = true; break; }
    int off = 0;
    if (K > 0) {
      LR_CUDA(h, cudaMemcpy2DAsync(x.b.L, sizeof(double) * x.ldp, dst.U, sizeof(double) * ldo, sizeof(double) * rows, K,
                                   cudaMemcpyDeviceToDevice, stm), "stack");
      LR_CUDA(h, cudaMemcpy2DAsync(x.b.Rt, sizeof(double) * x.ldp, dst.V, sizeof(double) * ldo, sizeof(double) * rows, K,
                                   cudaMemcpyDeviceToDevice, stm), "stack");
      LR_CUDA(h, launch_scale_copy(K, dst.s, 1.0, x.wts, stm), "weights");
      off = K;
      x.launches += 1;
    }
    while (off < KMAX && ti < tv.size()) {
      const Term& t = tv[ti];
      const int c = std::min(KMAX - off, t.r - tj);
      LR_CUDA(h, cudaMemcpy2DAsync(x.b.L + (size_t)off * x.ldp, sizeof(double) * x.ldp, t.U + (size_t)tj * t.ld,
                                   sizeof(double) * t.ld, sizeof(double) * rows, c, cudaMemcpyDeviceToDevice, stm),
             "stack");
      LR_CUDA(h, cudaMemcpy2DAsync(x.b.Rt + (size_t)off * x.ldp, sizeof(double) * x.ldp, t.V + (size_t)tj * t.ld,
                                   sizeof(double) * t.ld, sizeof(double) * rows, c, cudaMemcpyDeviceToDevice, stm),
             "stack");
      LR_CUDA(h, launch_scale_copy(c, t.s ? t.s + tj : nullptr, t.coef, x.wts + off, stm), "weights");
      x.launches += 1;
      off += c;
      tj += c;
      if (tj == t.r) { ++ti; tj = 0; }
    }
    const bool last = ti == tv.size();
    double sig = 0.0;
    lr_status s = qr_round(h, x.b, x.b.L, x.b.Rt, x.ldp, rows, off, x.wts, last ? x.eps : x.eps / 4.0, KMAX, dst.U,
                           dst.V, dst.s, ldo, 0, false, &K, &sig, single ? abs_tol : abs_tol / 2.0);
    x.launches += kQrRoundLaunches;
    if (s != LR_OK && s != LR_ENOCONV) return s;
  }
  dst.r = K;
  return LR_OK;
}

lr_status sum_round(StokesCtx& x, int rows, std::initializer_list<Term> terms, LrDev& dst, int ldo,
                    double abs_tol = 0.0) {
  return sum_round(x, rows, std::vector<Term>(terms), dst, ldo, abs_tol);
}

lr_status norm2_of(StokesCtx& x, const LrDev& a, double* out) {
  *out = 0.0;
  if (a.r == 0) return LR_OK;
  LR_CUDA(x.h, cudaMemcpyAsync(x.hbuf, a.s, sizeof(double) * a.r, cudaMemcpyDeviceToHost, x.h->stream), "copy");
  LR_CUDA(x.h, cudaStreamSynchronize(x.h->stream), "sync");
  for (int k = 0; k < a.r; ++k) *out += x.hbuf[k] * x.hbuf[k];
  return LR_OK;
}

// <A, B> = sum_kl sa_k sb_l (Ua^T Ub)_kl (Va^T Vb)_kl, float64.
lr_status inner(StokesCtx& x, int rows, const LrDev& a, const LrDev& b, double* out) {
  *out = 0.0;
  if (a.r == 0 || b.r == 0) return LR_OK;
  cudaStream_t stm = x.h->stream;
  LR_CUDA(x.h, launch_cross_gram(a.U, x.ldp, b.U, x.ldp, rows, a.r, b.r, x.gm0, x.xpart, stm), "gram");
  LR_CUDA(x.h, launch_cross_gram(a.V, x.ldp, b.V, x.ldp, rows, a.r, b.r, x.gm1, x.xpart, stm), "gram");
  x.launches += 4;
  double* hg0 = x.hbuf;
  double* hg1 = x.hbuf + KMAX * KMAX;
  double* hsa = x.hbuf + 2 * KMAX * KMAX;
  double* hsb = hsa + KMAX;
  const size_t gb = sizeof(double) * a.r * b.r;
  LR_CUDA(x.h, cudaMemcpyAsync(hg0, x.gm0, gb, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(x.h, cudaMemcpyAsync(hg1, x.gm1, gb, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(x.h, cudaMemcpyAsync(hsa, a.s, sizeof(double) * a.r, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(x.h, cudaMemcpyAsync(hsb, b.s, sizeof(double) * b.r, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(x.h, cudaStreamSynchronize(stm), "sync");
  double acc = 0.0;
  for (int l = 0; l < b.r; ++l)
    for (int k = 0; k < a.r; ++k) acc += hsa[k] * hsb[l] * hg0[k + l * a.r] * hg1[k + l * a.r];
  *out = acc;
  return LR_OK;
}

// W = A^-1 (B_x X, B_y X) for a pressure X: the d = 2 velocity solves of a
// Schur product, batched.  *rx, *ry: the ranks of the two solutions.
lr_status velocity_solves(StokesCtx& x, const lr_mat* rhs, int* rx, int* ry) {
  lr_handle h = x.h;
  const int m = x.n - 1;
  lr_mat sol[2];
  for (int k = 0; k < 2; ++k) sol[k] = {m, m, 0, KMAX, x.ldv, x.WU[k], x.Ws[k], x.WV[k]};
  std::vector<Plan*> plans(2, x.plan);
  lr_status per[2] = {LR_OK, LR_OK};
  lr_status s = x.oin.prec == LR_MIXED ? solve2d_batched<float>(h, 2, rhs, sol, x.oin, plans, per, false)
                                       : solve2d_batched<double>(h, 2, rhs, sol, x.oin, plans, per, false);
  x.launches += h->info.launches;
  if (s == LR_ENONFINITE && x.oin.prec == LR_MIXED) {
    // A float32 solve broke down (noise-level pivots on a direction whose
    // solution float32 cannot resolve): solve that problem again in float64.
    s = LR_OK;
    for (int k = 0; k < 2; ++k) {
      if (per[k] != LR_ENONFINITE) continue;
      lr_options o64 = x.oin;
      o64.prec = LR_FP64;
      const lr_status s2 = solve2d<double>(h, &rhs[k], &sol[k], o64, x.plan);
      if (s2 != LR_OK && s2 != LR_ENOCONV) return s2;
      ++x.escalations;
    }
  }
  if (s != LR_OK && s != LR_ENOCONV) return s;
  *rx = sol[0].r;
  *ry = sol[1].r;
  return LR_OK;
}

lr_status grad_solve(StokesCtx& x, const LrDev& X, int* rx, int* ry) {
  lr_handle h = x.h;
  cudaStream_t stm = h->stream;
  const int n = x.n, m = n - 1;
  if (X.r == 0) { *rx = *ry = 0; return LR_OK; }
  // The directions shrink with the residual: solve at unit scale (divide by
  // sigma_0 of X, multiply the solutions back) so float32 solves stay far
  // from the ends of their range.
  LR_CUDA(h, cudaMemcpyAsync(x.hbuf, X.s, sizeof(double), cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(h, cudaStreamSynchronize(stm), "sync");
  const double s0 = x.hbuf[0] > 0.0 ? x.hbuf[0] : 1.0;
  const double c = n / 4.0 / s0;  // 1 / (4h), at unit scale
  LR_CUDA(h, launch_gh(OP_G, n, X.U, x.ldp, X.r, X.s, c, x.RU[0], x.ldv, stm), "grad");
  LR_CUDA(h, launch_gh(OP_H, n, X.V, x.ldp, X.r, nullptr, 1.0, x.RV[0], x.ldv, stm), "grad");
  LR_CUDA(h, launch_gh(OP_H, n, X.U, x.ldp, X.r, X.s, c, x.RU[1], x.ldv, stm), "grad");
  LR_CUDA(h, launch_gh(OP_G, n, X.V, x.ldp, X.r, nullptr, 1.0, x.RV[1], x.ldv, stm), "grad");
  x.launches += 4;
  lr_mat rhs[2];
  for (int k = 0; k < 2; ++k) rhs[k] = {m, m, X.r, X.r, x.ldv, x.RU[k], nullptr, x.RV[k]};
  lr_status s = velocity_solves(x, rhs, rx, ry);
  if (s != LR_OK) return s;
  LR_CUDA(h, launch_scale_copy(*rx, x.Ws[0], s0, x.Ws[0], stm), "rescale");
  LR_CUDA(h, launch_scale_copy(*ry, x.Ws[1], s0, x.Ws[1], stm), "rescale");
  x.launches += 2;
  return LR_OK;
}

// dst = round(B^T W) for the velocity solutions of grad_solve (ranks rx, ry):
// the sum of (G^T Wx c)(H^T Zx)^T diag(sx) and (H^T Wy c)(G^T Zy)^T diag(sy),
// c = 1 / (4h), built in x.b.XU / XV and x.b.FU / FV.
lr_status div_round(StokesCtx& x, int rx, int ry, LrDev& dst, double abs_tol = 0.0) {
  lr_handle h = x.h;
  cudaStream_t stm = h->stream;
  const int n = x.n;
  const double c = n / 4.0;
  LR_CUDA(h, launch_gh(OP_GT, n, x.WU[0], x.ldv, rx, nullptr, 1.0, x.b.XU, x.ldp, stm), "div");
  LR_CUDA(h, launch_gh(OP_HT, n, x.WV[0], x.ldv, rx, nullptr, 1.0, x.b.XV, x.ldp, stm), "div");
  LR_CUDA(h, launch_gh(OP_HT, n, x.WU[1], x.ldv, ry, nullptr, 1.0, x.b.FU, x.ldp, stm), "div");
  LR_CUDA(h, launch_gh(OP_GT, n, x.WV[1], x.ldv, ry, nullptr, 1.0, x.b.FV, x.ldp, stm), "div");
  x.launches += 4;
  return sum_round(x, n, {{x.b.XU, x.Ws[0], x.b.XV, rx, x.ldp, c}, {x.b.FU, x.Ws[1], x.b.FV, ry, x.ldp, c}}, dst,
                   x.ldp, abs_tol);
}

lr_status copy_lr(StokesCtx& x, int rows, const LrDev& a, LrDev& dst) {
  dst.r = a.r;
  if (a.r == 0) return LR_OK;
  cudaStream_t stm = x.h->stream;
  const size_t bytes = sizeof(double) * (size_t)x.ldp * a.r;
  (void)rows;
  LR_CUDA(x.h, cudaMemcpyAsync(dst.U, a.U, bytes, cudaMemcpyDeviceToDevice, stm), "copy");
  LR_CUDA(x.h, cudaMemcpyAsync(dst.V, a.V, bytes, cudaMemcpyDeviceToDevice, stm), "copy");
  LR_CUDA(x.h, cudaMemcpyAsync(dst.s, a.s, sizeof(double) * a.r, cudaMemcpyDeviceToDevice, stm), "copy");
  return LR_OK;
}

// coef * <X, 1 1^T> / n^2 and coef * <X, c c^T> / n^2 (c = (-1)^i): the
// weights of the two kernel modes (as the columns 1 and c of x.E) in X.
lr_status kernel_coeffs(StokesCtx& x, const LrDev& X, double coef, double* a, double* b) {
  *a = *b = 0.0;
  if (X.r == 0) return LR_OK;
  lr_handle h = x.h;
  cudaStream_t stm = h->stream;
  const int n = x.n, r = X.r;
  LR_CUDA(h, launch_colsums(X.U, x.ldp, n, r, x.cs, stm), "colsums");
  LR_CUDA(h, launch_colsums(X.V, x.ldp, n, r, x.cs + 2 * KMAX, stm), "colsums");
  LR_CUDA(h, cudaMemcpyAsync(x.hbuf, x.cs, sizeof(double) * 4 * KMAX, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(h, cudaMemcpyAsync(x.hbuf + 4 * KMAX, X.s, sizeof(double) * r, cudaMemcpyDeviceToHost, stm), "copy");
  LR_CUDA(h, cudaStreamSynchronize(stm), "sync");
  x.launches += 2;
  const double* cu = x.hbuf;             // [sum U_k, sum (-1)^i U_k]
  const double* cw = x.hbuf + 2 * KMAX;  // the same for V
  const double* sp = x.hbuf + 4 * KMAX;
  for (int k = 0; k < r; ++k) {
    *a += sp[k] * cu[k] * cw[k];
    *b += sp[k] * cu[r + k] * cw[r + k];
  }
  *a *= coef / ((double)n * n);
  *b *= coef / ((double)n * n);
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Low-rank 3D solve in Tucker format (Section 3, Eq. flr:tucker; Sections 4.1
// and 4.2 in three dimensions): forward DST of the three factors, Tucker
// fibre cross of Xh = Fh / (mu_i + mu_j + mu_k) (kernels in tucker.cu), the
// higher-order SVD of its core (shifted Cholesky QR of each unfolding and the
// rounding core), inverse DST of the kept factors.  float64 throughout.
// ---------------------------------------------------------------------------

// Output t (1-based) of splitmix64 started at state seed (Steele, Lea and
// Flood 2014): the probe positions of the 3D cross.
unsigned long long splitmix64_at(unsigned long long seed, unsigned long long t) {
  unsigned long long z = seed + t * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int kT3ProbeRounds = 4;

int q_cap(int p) { return p < 1 ? 1 : p; }

lr_status solve3d_tucker(lr_handle h, const lr_tucker* rhs, lr_tucker* sol, const lr_options& o) {
  cudaStream_t stm = h->stream;
  // LR_MIXED: float32 transforms and float32 Jacobi in the rounding cores of
  // the higher-order SVD; the cross in float64
  const bool mixed = o.prec == LR_MIXED;
  Plan* plan[3];
  int n[3], r[3], ldq[3];
  int nmax = 0;
  size_t Mmax = 0;
  for (int k = 0; k < 3; ++k) {
    n[k] = rhs->n[k];
    r[k] = rhs->r[k];
    ldq[k] = n[k] + (n[k] & 1);
    nmax = std::max(nmax, n[k]);
    lr_status s = get_plan(h, n[k], &plan[k]);
    if (s != LR_OK) return s;
    Mmax = std::max(Mmax, (size_t)1 << plan[k]->logM);
  }
  const int probes = std::max(0, o.probes);
  const int maxjobs = 3 * (probes + T3P * T3P);
  const int lda = T3P * T3P;  // unfoldings: at most 64 x 64 rows
  const size_t cube = sizeof(double) * (size_t)T3P * T3P * T3P;
  T3Dev d{};
  double *T1 = nullptr, *T2 = nullptr, *E = nullptr, *ident = nullptr, *W[3] = {}, *sig[3] = {}, *XU[3] = {};
  int *jobs = nullptr, *pam = nullptr;
  double* pn2 = nullptr;
  RefineBufs b3[3];
  auto layout = [&](Carve& c) {
    for (int k = 0; k < 3; ++k) {
      d.Uh[k] = c.take<double>(sizeof(double) * (size_t)ldq[k] * r[k]);
      d.Q[k] = c.take<double>(sizeof(double) * (size_t)ldq[k] * T3P);
      d.e[k] = c.take<double>(sizeof(double) * ldq[k]);
      d.v[k] = c.take<double>(sizeof(double) * ldq[k]);
      d.inI[k] = c.take<unsigned char>(n[k]);
      d.Minv[k] = c.take<double>(sizeof(double) * T3P * T3P);
      d.I[k] = c.take<int>(sizeof(int) * T3P);
      d.h[k] = c.take<double>(sizeof(double) * (T3P + 1));
      d.y[k] = c.take<double>(sizeof(double) * T3P);
      W[k] = c.take<double>(sizeof(double) * KMAX * KMAX);
    }
    d.C = c.take<double>(cube);
    T1 = c.take<double>(cube);
    T2 = c.take<double>(cube);
    E = c.take<double>(cube);
    d.st = c.take<T3State>(sizeof(T3State));
    jobs = c.take<int>(sizeof(int) * 3 * (size_t)maxjobs);
    pn2 = c.take<double>(sizeof(double) * (size_t)maxjobs);
    pam = c.take<int>(sizeof(int) * (size_t)maxjobs);
    ident = c.take<double>(sizeof(double) * KMAX * KMAX);
    for (int k = 0; k < 3; ++k) {
      sig[k] = c.take<double>(sizeof(double) * KMAX);
      XU[k] = c.take<double>(sizeof(double) * (size_t)ldq[k] * KMAX);
      carve_refine(c, b3[k], lda, lda);  // Cholesky QR of unfolding k (XU: the unfolding, L, Lb: lda x 64)
    }
  };
  Carve sizing;
  layout(sizing);
  if (sizing.off > h->ws5_bytes) {
    const lr_status sg = grow_ws(h, &h->ws5, &h->ws5_bytes, sizing.off, "3D workspace");
    if (sg != LR_OK) return sg;
  }
  if (!h->h_big && cudaMallocHost(&h->h_big, sizeof(double) * (2 * KMAX * KMAX + 4 * KMAX)) != cudaSuccess) {
    cudaGetLastError();
    h->h_big = nullptr;
    return fail(h, LR_ENOMEM, "pinned buffer");
  }
  Carve cv;
  cv.base = static_cast<char*>(h->ws5);
  layout(cv);
  for (int k = 0; k < 3; ++k) {
    d.n[k] = n[k];
    d.r[k] = r[k];
    d.ldu[k] = ldq[k];
    d.ldq[k] = ldq[k];
    d.mu[k] = plan[k]->sym_a64[LR_OP_5PT];
  }
  d.G = rhs->G;
  int launches = 0;
  // forward transforms of the factors
  lr_status s = ensure_ws(h, Mmax > (size_t)kSmallM ? Mmax * 2 * (size_t)KMAX * sizeof(cpx<double>) + 256 : 256);
  if (s != LR_OK) return s;
  for (int k = 0; k < 3; ++k) {
    ColumnSet cs;
    cs.in[0] = rhs->U[k];
    cs.ld_in[0] = rhs->ld[k];
    cs.out[0] = const_cast<double*>(d.Uh[k]);
    cs.ld_out[0] = ldq[k];
    cs.ncol[0] = r[k];
    LR_CUDA(h, mixed ? launch_dst<float>(*plan[k], cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm)
                     : launch_dst<double>(*plan[k], cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm),
            "3D: forward");
    ++launches;
  }
  // state
  for (int k = 0; k < 3; ++k) {
    LR_CUDA(h, cudaMemsetAsync(d.inI[k], 0, n[k], stm), "3D: init");
    LR_CUDA(h, cudaMemsetAsync(d.Minv[k], 0, sizeof(double) * T3P * T3P, stm), "3D: init");
  }
  T3State* hs = reinterpret_cast<T3State*>(h->h_big);
  std::memset(hs, 0, sizeof(T3State));
  hs->rho0 = -1.0;
  LR_CUDA(h, cudaMemcpyAsync(d.st, hs, sizeof(T3State), cudaMemcpyHostToDevice, stm), "3D: init");
  const double tol = 0.1 * o.aca_tol_factor * o.eps;
  auto read_state = [&]() -> lr_status {
    LR_CUDA(h, cudaMemcpyAsync(hs, d.st, sizeof(T3State), cudaMemcpyDeviceToHost, stm), "3D: state");
    LR_CUDA(h, cudaStreamSynchronize(stm), "3D: cross");
    if (hs->status) return fail(h, static_cast<lr_status>(hs->status), "3D: non-finite value in the cross");
    return LR_OK;
  };
  const size_t P = T3P, P2 = (size_t)T3P * T3P;
  auto mp = [&](const double* in, std::array<size_t, 3> is, double* out, std::array<size_t, 3> os,
                std::array<int, 3> od, int mode, int K, const double* A, const int* rowmap, int ars, int acs,
                int divlam) -> cudaError_t {
    T3ModeProd a;
    a.in = in;
    a.out = out;
    for (int k = 0; k < 3; ++k) { a.is[k] = (int)is[k]; a.os[k] = (int)os[k]; a.od[k] = od[k]; }
    a.mode = mode;
    a.K = K;
    a.A = A;
    a.rowmap = rowmap;
    a.ars = ars;
    a.acs = acs;
    a.divlam = divlam;
    ++launches;
    return launch_t3_modeprod(a, d, stm);
  };
  bool converged = false;
  std::vector<int> hjobs;
  std::vector<int> hI(3 * T3P);
  // One step of the cross as a fixed launch sequence (every size it depends
  // on is read from the device state), captured once as a CUDA graph: the
  // pivot search, the pivot, the basis updates, the core C = Xh(I1, I2, I3)
  // x_k M_k (Fh on the index grid by three mode products of G, the last one
  // divided by Lambda, then the inverses) and the step test.
  auto step_body = [&](cudaStream_t sq) -> cudaError_t {
    cudaError_t e;
    if ((e = launch_t3_search(d, sq)) != cudaSuccess) return e;
    if ((e = launch_t3_pivot(d, sq)) != cudaSuccess) return e;
    if ((e = launch_t3_basis_update(d, nmax, sq)) != cudaSuccess) return e;
    const std::array<size_t, 3> sg{(size_t)r[1] * r[2], (size_t)r[2], 1}, sc{1, P, P2};
    const int P0 = -1, P1 = -2, P2d = -3;  // device basis sizes p_0, p_1, p_2
    auto prod = [&](const double* in, std::array<size_t, 3> is, double* out, std::array<int, 3> od, int mode, int K,
                    const double* Am, const int* rowmap, int acs, int divlam) {
      T3ModeProd a;
      a.in = in;
      a.out = out;
      for (int k = 0; k < 3; ++k) { a.is[k] = (int)is[k]; a.os[k] = (int)sc[k]; a.od[k] = od[k]; }
      a.mode = mode;
      a.K = K;
      a.A = Am;
      a.rowmap = rowmap;
      a.ars = 1;
      a.acs = acs;
      a.divlam = divlam;
      a.skip_negl = 1;
      return launch_t3_modeprod(a, d, sq);
    };
    if ((e = prod(d.G, sg, T1, {P0, r[1], r[2]}, 0, r[0], d.Uh[0], d.I[0], ldq[0], 0)) != cudaSuccess) return e;
    if ((e = prod(T1, sc, T2, {P0, P1, r[2]}, 1, r[1], d.Uh[1], d.I[1], ldq[1], 0)) != cudaSuccess) return e;
    if ((e = prod(T2, sc, E, {P0, P1, P2d}, 2, r[2], d.Uh[2], d.I[2], ldq[2], 1)) != cudaSuccess) return e;
    if ((e = prod(E, sc, T1, {P0, P1, P2d}, 0, P0, d.Minv[0], nullptr, T3P, 0)) != cudaSuccess) return e;
    if ((e = prod(T1, sc, T2, {P0, P1, P2d}, 1, P1, d.Minv[1], nullptr, T3P, 0)) != cudaSuccess) return e;
    if ((e = prod(T2, sc, d.C, {P0, P1, P2d}, 2, P2d, d.Minv[2], nullptr, T3P, 0)) != cudaSuccess) return e;
    return launch_t3_decide(d, tol, sq);
  };
  char key[512];
  snprintf(key, sizeof key, "t3step|%p,%zu|%p|%d,%d,%d|%d,%d,%d|%.17g|%d|%d", h->ws5, h->ws5_bytes, (void*)rhs->G,
           n[0], n[1], n[2], r[0], r[1], r[2], tol, nmax, probes);
  for (int step = 0; step < o.rmax; ++step) {
    if ((s = run_maybe_graph(h, true, key, step_body)) != LR_OK) return s;
    launches += 16;
    if ((s = read_state()) != LR_OK) return s;
    if (hs->done) { converged = hs->converged != 0; break; }
    if (hs->small < 2) continue;
    if (probes == 0 || hs->probe_rounds >= kT3ProbeRounds) { converged = true; break; }
    // probe round: random fibres of every mode, then the fibres through the
    // other two modes' index sets
    for (int k = 0; k < 3; ++k)
      if (hs->p[k] > 0)
        LR_CUDA(h, cudaMemcpyAsync(hI.data() + k * T3P, d.I[k], sizeof(int) * hs->p[k], cudaMemcpyDeviceToHost, stm),
                "3D: indices");
    LR_CUDA(h, cudaStreamSynchronize(stm), "3D: indices");
    const unsigned long long seed = o.seed + (unsigned long long)hs->probe_rounds;
    hjobs.clear();
    T3ProbeCounts cnt{};
    for (int m = 0; m < 3; ++m) {
      const int oa = m == 0 ? 1 : 0, ob = m == 2 ? 1 : 2;
      for (int t = 0; t < probes; ++t) {
        const unsigned long long z = splitmix64_at(seed, (unsigned long long)(m * probes + t + 1));
        hjobs.insert(hjobs.end(), {m, (int)((z >> 32) % (unsigned long long)n[oa]),
                                   (int)((z & 0xFFFFFFFFull) % (unsigned long long)n[ob])});
      }
      cnt.nrand[m] = probes;
      for (int x = 0; x < hs->p[oa]; ++x)
        for (int y = 0; y < hs->p[ob]; ++y) hjobs.insert(hjobs.end(), {m, hI[oa * T3P + x], hI[ob * T3P + y]});
      cnt.ncross[m] = hs->p[oa] * hs->p[ob];
    }
    const int nfib = (int)hjobs.size() / 3;
    LR_CUDA(h, cudaMemcpyAsync(jobs, hjobs.data(), sizeof(int) * hjobs.size(), cudaMemcpyHostToDevice, stm), "3D: jobs");
    LR_CUDA(h, launch_t3_probe(d, nfib, jobs, pn2, pam, stm), "3D: probes");
    LR_CUDA(h, launch_t3_probe_reduce(d, jobs, pn2, pam, cnt, tol, stm), "3D: probes");
    launches += 2;
    if ((s = read_state()) != LR_OK) return s;
    if (hs->done) { converged = true; break; }
  }
  // Rounding: higher-order SVD of the core.  For each mode the unfolding's
  // transpose C_(m)^T = Q R (shifted Cholesky QR); the rounding core on
  // M = I R^T gives the left singular vectors W_m of C_(m) and its singular
  // values, truncated with a tail <= eps ||C|| / sqrt(3).
  const int p[3] = {hs->p[0], hs->p[1], hs->p[2]};
  {
    std::vector<double> id(KMAX * KMAX, 0.0);
    for (int i = 0; i < KMAX; ++i) id[i + i * KMAX] = 1.0;
    LR_CUDA(h, cudaMemcpyAsync(ident, id.data(), sizeof(double) * id.size(), cudaMemcpyHostToDevice, stm), "3D: identity");
    LR_CUDA(h, cudaStreamSynchronize(stm), "3D: identity");
  }
  int R[3] = {0, 0, 0};
  bool cut = false;
  if (p[0] * p[1] * p[2] > 0) {
    // the three modes are independent: one stream each, with their own scratch
    if ((s = ensure_batch_streams(h)) != LR_OK) return s;
    LR_CUDA(h, cudaEventRecord(h->bfork, stm), "3D: fork");
    for (int m = 0; m < 3; ++m) {
      cudaStream_t sm = h->bstreams[m];
      const RefineBufs& b = b3[m];
      double* A = b.XU;  // lda x 64
      LR_CUDA(h, cudaStreamWaitEvent(sm, h->bfork, 0), "3D: fork");
      const int oa = m == 0 ? 1 : 0, ob = m == 2 ? 1 : 2;
      const int q = p[m], rows = p[oa] * p[ob];
      LR_CUDA(h, launch_t3_unfold(d, m, q * rows, A, lda, sm), "3D: unfold");
      const double shift = 11.0 * ((double)rows * q + (double)q * (q + 1)) * (DBL_EPSILON / 2) * q;
      const double* X = A;
      for (int step = 0; step < kQrSteps; ++step) {
        LR_CUDA(h, launch_gram(X, rows, lda, q, b.G0, q, b.part, h->num_sms, sm), "3D: gram");
        CholQrArgs a;
        a.G[0] = b.G0; a.G[1] = b.G0;
        a.T[0] = b.T0; a.T[1] = b.T1;
        a.Racc[0] = b.Ra0; a.Racc[1] = b.Ra1;
        a.qout = b.qout;
        a.q = q;
        a.first = step == 0;
        a.shift = step < kQrShiftedSteps ? shift : 0.0;
        a.floor_rel = 0.0;
        LR_CUDA(h, launch_cholqr_step(a, sm), "3D: cholesky qr");
        launches += 3;
        if (step + 1 < kQrSteps) {
          double* Y = (step & 1) ? b.L : b.Lb;
          LR_CUDA(h, (launch_rotate<double, double>(X, lda, rows, nullptr, q, b.T0, false, &b.qout[0], Y, lda, sm)), "3D: qr");
            X = Y;
        }
      }
      LR_CUDA(h, cudaMemsetAsync(b.st, 0, sizeof(SolveState), sm), "state reset");
      if (mixed) {
        // float32 coefficient matrices in the (larger) float64 buffers, widened into W
        CoreArgs<float> co;
        co.GC = ident; co.GR = b.Ra0; co.ldg = KMAX; co.d = nullptr;
        co.k_dev = nullptr; co.k_host = q;
        co.eps = o.eps / std::sqrt(3.0); co.rmax_out = std::min(sol->rmax[m], KMAX);
        co.Tc = reinterpret_cast<float*>(b.Tc); co.Tr = reinterpret_cast<float*>(b.Tr);
        co.s_out = sig[m]; co.st = b.st;
        co.tri_given = 1;
        LR_CUDA(h, launch_core<float>(co, true, sm), "3D: core SVD");
        LR_CUDA(h, launch_t3_widen(reinterpret_cast<const float*>(b.Tc), W[m], KMAX * KMAX, sm), "3D: W");
      } else {
        CoreArgs<double> co;
        co.GC = ident; co.GR = b.Ra0; co.ldg = KMAX; co.d = nullptr;
        co.k_dev = nullptr; co.k_host = q;
        co.eps = o.eps / std::sqrt(3.0); co.rmax_out = std::min(sol->rmax[m], KMAX);
        co.Tc = b.Tc; co.Tr = b.Tr; co.s_out = sig[m]; co.st = b.st;
        co.tri_given = 1;
        LR_CUDA(h, launch_core<double>(co, false, sm), "3D: core SVD");
        LR_CUDA(h, cudaMemcpyAsync(W[m], b.Tc, sizeof(double) * KMAX * KMAX, cudaMemcpyDeviceToDevice, sm), "3D: W");
      }
      // kept factor Q_m W_m (its rank read on the device)
      LR_CUDA(h, (launch_rotate<double, double>(d.Q[m], ldq[m], n[m], nullptr, q, W[m], false, &b.st->rank, XU[m], ldq[m], sm)), "3D: rot");
      launches += 3;
      LR_CUDA(h, cudaEventRecord(h->bjoin[m], sm), "3D: join");
      LR_CUDA(h, cudaStreamWaitEvent(stm, h->bjoin[m], 0), "3D: join");
    }
    // inverse transforms of the kept factors into the caller's U_m (on the
    // handle's stream: they share the transform scratch)
    for (int m = 0; m < 3; ++m) {
      ColumnSet cs;
      cs.in[0] = XU[m];
      cs.ld_in[0] = ldq[m];
      cs.out[0] = sol->U[m];
      cs.ld_out[0] = sol->ld[m];
      cs.ncol[0] = std::min(sol->rmax[m], q_cap(p[m]));
      cs.dyn_count = &b3[m].st->rank;
      LR_CUDA(h, mixed ? launch_dst<float>(*plan[m], cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm)
                       : launch_dst<double>(*plan[m], cs, IoType::F64, IoType::F64, h->ws, h->num_sms, stm),
              "3D: inverse");
      ++launches;
    }
    SolveState* hst = reinterpret_cast<SolveState*>(h->h_big + 512);
    for (int m = 0; m < 3; ++m)
      LR_CUDA(h, cudaMemcpyAsync(hst + m, b3[m].st, sizeof(SolveState), cudaMemcpyDeviceToHost, stm), "state copy");
    LR_CUDA(h, cudaStreamSynchronize(stm), "3D: rounding");
    for (int m = 0; m < 3; ++m) {
      if (hst[m].status) return fail(h, static_cast<lr_status>(hst[m].status), kNonFiniteMsg);
      R[m] = hst[m].rank;
      if (hst[m].cut) cut = true;
    }
  }
  if (R[0] * R[1] * R[2] > 0) {
    // G_out = C x_1 W_1^T x_2 W_2^T x_3 W_3^T, written in C order
    const std::array<size_t, 3> sc{1, P, P2};
    const std::array<size_t, 3> so{(size_t)R[1] * R[2], (size_t)R[2], 1};
    LR_CUDA(h, mp(d.C, sc, T1, sc, {R[0], p[1], p[2]}, 0, p[0], W[0], nullptr, KMAX, 1, 0), "3D: core out");
    LR_CUDA(h, mp(T1, sc, T2, sc, {R[0], R[1], p[2]}, 1, p[1], W[1], nullptr, KMAX, 1, 0), "3D: core out");
    LR_CUDA(h, mp(T2, sc, sol->G, so, {R[0], R[1], R[2]}, 2, p[2], W[2], nullptr, KMAX, 1, 0), "3D: core out");
  } else {
    R[0] = R[1] = R[2] = 0;
  }
  LR_CUDA(h, cudaStreamSynchronize(stm), "3D solve");
  for (int k = 0; k < 3; ++k) sol->r[k] = R[k];
  h->info = lr_info{};
  h->info.aca_steps = hs->steps;
  h->info.probe_rounds = hs->probe_rounds;
  h->info.converged = converged ? 1 : 0;
  h->info.rank = std::max(R[0], std::max(R[1], R[2]));
  h->info.cut = cut ? 1 : 0;
  h->info.launches = launches;
  h->info.norm_est = hs->nrmC;
  // lr_get_info reports from the solve state record
  SolveState& ss = *h->h_state;
  ss.k = hs->steps;
  ss.rank = h->info.rank;
  ss.converged = h->info.converged;
  ss.cut = h->info.cut;
  ss.probe_rounds = hs->probe_rounds;
  ss.zero_rows = 0;
  ss.norm2 = hs->nrmC * hs->nrmC;
  if (cut) return fail(h, LR_ENOCONV, "a Tucker rank exceeds sol->rmax; result truncated");
  if (!converged) return fail(h, LR_ENOCONV, "3D cross did not converge within rmax steps");
  return LR_OK;
}

// w = (B^T A^-1 B) v with the velocity solves and the rounding of B^T u at
// relative accuracy delta.  In LR_MIXED a product asked for below 1e-6 (what
// float32 solves resolve) runs its velocity solves in float64: with the
// relaxed accuracies of GMRES that is the first product of a cycle and the
// residuals of the restarts, the rest stays in float32.
lr_status schur_product(StokesCtx& x, const LrDev& v, LrDev& w, double delta) {
  const double e_in = x.oin.eps, e_r = x.eps;
  const lr_precision p_in = x.oin.prec;
  // velocity solves a tenth tighter than the product (B^T, a difference over
  // h, amplifies their high-frequency error)
  const double d_in = 0.1 * delta;
  if (x.oin.prec == LR_MIXED && d_in < 1e-6) x.oin.prec = LR_FP64;
  x.oin.eps = d_in;
  x.eps = delta;
  int rx = 0, ry = 0;
  lr_status s = grad_solve(x, v, &rx, &ry);
  if (s == LR_OK) s = div_round(x, rx, ry, w);
  x.oin.eps = e_in;
  x.oin.prec = p_in;
  x.eps = e_r;
  return s;
}

// Restarted inexact GMRES(kGmresRestart) on the Schur equation (Section 5: the
// paper's Stokes solver; adaptive accuracy of the products after Simoncini
// and Szyld 2003): the product with the j-th Krylov vector is formed at
// relative accuracy min(kGmresMaxDelta, tol ||r0|| / (2 ||r_j||)), exact early
// and relaxed as the residual falls; the new vector w - sum_i h_ij V_i is formed
// by modified Gram-Schmidt, each step rounded at that accuracy (kernel modes
// of the pressure projected out at the last); the small least-squares problem
// is solved by Givens rotations on the host; at a restart p <- p + y_i V_i is
// rounded at eps term by term and the residual rhs - S p recomputed.  x.R holds the
// right-hand side B^T A^-1 f; the result goes to x.P.
lr_status stokes_gmres(StokesCtx& x, double tol, int maxit, double nr0, int* it_out, double* res_out,
                       double* history) {
  const int n = x.n, m = kGmresRestart;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), y(m, 0.0);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i + (size_t)j * (m + 1)]; };
  int it = 0;
  double res = nr0;
  lr_status s;  // x.P: the initial guess (empty, or a resumed pressure)
  // Only a cut of the pressure update counts (x.cut on return): a Krylov
  // vector or a product that needed more than 64 columns only changes the
  // space searched, and the result is certified by its true residual.
  const bool cut_in = x.cut;
  bool pcut = false;
  auto scale_vec = [&](LrDev& v, double c) -> lr_status {
    if (v.r > 0) LR_CUDA(x.h, launch_scale_copy(v.r, v.s, c, v.s, x.h->stream), "scale");
    return LR_OK;
  };
  while (it < maxit) {
    // r = rhs - S p, kernel modes projected out
    if (x.P.r == 0) {
      if ((s = copy_lr(x, n, x.R, x.K[0])) != LR_OK) return s;
    } else {
      if ((s = schur_product(x, x.P, x.Q, 0.1 * x.eps)) != LR_OK) return s;
      double ka = 0.0, kb = 0.0, qa = 0.0, qb = 0.0;
      if ((s = kernel_coeffs(x, x.R, 1.0, &ka, &kb)) != LR_OK) return s;
      if ((s = kernel_coeffs(x, x.Q, -1.0, &qa, &qb)) != LR_OK) return s;
      if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.Q.U, x.Q.s, x.Q.V, x.Q.r, x.ldp, -1.0},
                                {x.E, nullptr, x.E, 1, x.ldp, -(ka + qa)},
                                {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -(kb + qb)}},
                         x.K[0], x.ldp, 0.1 * x.eps * nr0)) != LR_OK)
        return s;
    }
    double b2 = 0.0;
    if ((s = norm2_of(x, x.K[0], &b2)) != LR_OK) return s;
    const double beta = std::sqrt(b2);
    res = beta;
    if (!(beta > tol * nr0)) break;
    if ((s = scale_vec(x.K[0], 1.0 / beta)) != LR_OK) return s;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    while (j < m && it < maxit) {
      const double delta = std::min(kGmresMaxDelta, 0.5 * tol * nr0 / res);
      if ((s = schur_product(x, x.K[j], x.Q, delta)) != LR_OK) return s;
      // modified Gram-Schmidt, each subtraction rounded at delta (a single sum
      // of all terms has partial sums of far higher rank than the result);
      // the last one also removes the kernel modes
      const double e_r = x.eps;
      x.eps = delta;
      for (int i = 0; i <= j && s == LR_OK; ++i) {
        if ((s = inner(x, n, x.Q, x.K[i], &Hij(i, j))) != LR_OK) break;
        std::vector<Term> terms;
        terms.push_back({x.Q.U, x.Q.s, x.Q.V, x.Q.r, x.ldp, 1.0});
        terms.push_back({x.K[i].U, x.K[i].s, x.K[i].V, x.K[i].r, x.ldp, -Hij(i, j)});
        LrDev& dst = i == j ? x.K[j + 1] : x.T;
        if (i == j) {
          double ka = 0.0, kb = 0.0;
          if ((s = kernel_coeffs(x, x.Q, -1.0, &ka, &kb)) != LR_OK) break;
          terms.push_back({x.E, nullptr, x.E, 1, x.ldp, ka});
          terms.push_back({x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, kb});
        }
        if ((s = sum_round(x, n, terms, dst, x.ldp)) != LR_OK) break;
        if (i != j) std::swap(x.Q, x.T);
      }
      x.eps = e_r;
      if (s != LR_OK) return s;
      double hn2 = 0.0;
      if ((s = norm2_of(x, x.K[j + 1], &hn2)) != LR_OK) return s;
      const double hn = std::sqrt(hn2);
      Hij(j + 1, j) = hn;
      if (hn > 0.0 && (s = scale_vec(x.K[j + 1], 1.0 / hn)) != LR_OK) return s;
      // Givens rotations: apply the previous ones to column j, then a new one
      for (int i = 0; i < j; ++i) {
        const double a = Hij(i, j), b = Hij(i + 1, j);
        Hij(i, j) = cs[i] * a + sn[i] * b;
        Hij(i + 1, j) = -sn[i] * a + cs[i] * b;
      }
      const double a = Hij(j, j), b = Hij(j + 1, j);
      const double rho = std::hypot(a, b);
      cs[j] = rho > 0.0 ? a / rho : 1.0;
      sn[j] = rho > 0.0 ? b / rho : 0.0;
      Hij(j, j) = rho;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      res = std::fabs(g[j + 1]);
      ++j;
      ++it;
      if (history) history[it] = res / nr0;
      if (res <= tol * nr0 || hn == 0.0) break;
    }
    // y = R^-1 g (upper triangular j x j), p <- round(p + sum_i y_i V_i)
    for (int i = j - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < j; ++l) acc -= Hij(i, l) * y[l];
      y[i] = Hij(i, i) != 0.0 ? acc / Hij(i, i) : 0.0;
    }
    for (int i = 0; i < j; ++i) {
      x.cut = false;
      if ((s = sum_round(x, n, {{x.P.U, x.P.s, x.P.V, x.P.r, x.ldp, 1.0},
                                {x.K[i].U, x.K[i].s, x.K[i].V, x.K[i].r, x.ldp, y[i]}},
                         x.T, x.ldp)) != LR_OK)
        return s;
      pcut = pcut || x.cut;
      std::swap(x.P, x.T);
    }
    if (res <= tol * nr0) {
      // the recursion's estimate met the tolerance: confirm on the true residual
      if ((s = schur_product(x, x.P, x.Q, 0.1 * x.eps)) != LR_OK) return s;
      double ka = 0.0, kb = 0.0, qa = 0.0, qb = 0.0;
      if ((s = kernel_coeffs(x, x.R, 1.0, &ka, &kb)) != LR_OK) return s;
      if ((s = kernel_coeffs(x, x.Q, -1.0, &qa, &qb)) != LR_OK) return s;
      if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.Q.U, x.Q.s, x.Q.V, x.Q.r, x.ldp, -1.0},
                                {x.E, nullptr, x.E, 1, x.ldp, -(ka + qa)},
                                {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -(kb + qb)}},
                         x.K[0], x.ldp, 0.1 * x.eps * nr0)) != LR_OK)
        return s;
      double t2 = 0.0;
      if ((s = norm2_of(x, x.K[0], &t2)) != LR_OK) return s;
      res = std::sqrt(t2);
      if (res <= tol * nr0) break;
      // otherwise the next cycle restarts from the true residual
    }
  }
  x.cut = cut_in || pcut;
  *it_out = it;
  *res_out = res;
  return LR_OK;
}

// Absolute rounding level of the CG residual and direction, in units of
// eps ||r0|| (the Schur product q: a tenth of it).
constexpr double kCgFloor = 0.3;

// The velocity solves of a Schur product, of the right-hand side B^T A^-1 f
// and of the final velocity carry their error through B^T, a difference over
// h, into the divergence: float32 solves (1e-6 at best) cannot deliver a
// product asked at a tenth of eps below 1e-6.  Those solves run in float64
// (the CG recursion and the final divergence then reach tol_div), the rest
// stay float32.  Restores the options on destruction.
struct VelocityPrecision {
  StokesCtx& x;
  lr_precision prec;
  double eps;
  VelocityPrecision(StokesCtx& xx, double eps_user) : x(xx), prec(xx.oin.prec), eps(xx.oin.eps) {
    if (x.oin.prec == LR_MIXED && 0.1 * eps_user < 1e-6) {
      x.oin.prec = LR_FP64;
      x.oin.eps = 0.1 * eps_user;
    }
  }
  ~VelocityPrecision() {
    x.oin.prec = prec;
    x.oin.eps = eps;
  }
};

lr_status stokes_uzawa(lr_handle h, int n, const lr_mat* f, const lr_mat* g, lr_mat* u, lr_mat* p, double tol,
                       int maxit, const lr_options& o, int* iters, double* resid, double* history) {
  StokesCtx x;
  x.h = h;
  x.n = n;
  x.ldp = n + (n & 1);
  x.ldv = (n - 1) + ((n - 1) & 1);
  x.eps = o.eps;
  x.oin = o;
  x.oin.flags = 0;
  x.oin.refine = -1;
  x.oin.op = LR_OP_SEMISTAGGERED;
  x.gmres = (o.flags & LR_FLAG_GMRES) != 0;
  // The velocity solves run at eps / 10: B^T is a difference over h and
  // amplifies the high-frequency part of their error, which the Schur
  // product q would otherwise carry into the CG recursion.  float32 solves:
  // below 1e-6 the float32 cross sits on its own rounding noise and does not
  // converge, so they run at 1e-6 at least.
  x.oin.eps = 0.1 * o.eps;
  if (o.prec == LR_MIXED && x.oin.eps < 1e-6) x.oin.eps = 1e-6;
  lr_status s = get_plan(h, n - 1, &x.plan);
  if (s != LR_OK) return s;
  Carve sizing;
  carve_stokes(sizing, x);
  if (sizing.off > h->ws4_bytes) {
    if ((s = grow_ws(h, &h->ws4, &h->ws4_bytes, sizing.off, "Stokes workspace")) != LR_OK) return s;
  }
  if (!h->h_big && cudaMallocHost(&h->h_big, sizeof(double) * (2 * KMAX * KMAX + 4 * KMAX)) != cudaSuccess) {
    cudaGetLastError();
    h->h_big = nullptr;
    return fail(h, LR_ENOMEM, "pinned buffer");
  }
  x.hbuf = h->h_big;
  Carve cv;
  cv.base = static_cast<char*>(h->ws4);
  carve_stokes(cv, x);
  cudaStream_t stm = h->stream;
  LR_CUDA(h, launch_kernel_modes(n, x.E, x.ldp, stm), "modes");
  // r0 = B^T A^-1 f
  int rx = 0, ry = 0;
  {
    VelocityPrecision vp(x, o.eps);
    if ((s = velocity_solves(x, f, &rx, &ry)) != LR_OK) return s;
  }
  if ((s = div_round(x, rx, ry, x.R)) != LR_OK) return s;
  // divergence right-hand side (B^T u = g): the Schur right-hand side is
  // B^T A^-1 f - g (Eq. flr:schur with -g); g's components along the kernel
  // modes cannot be met and are dropped
  double ga = 0.0, gb = 0.0;
  if (g && g->r > 0) {
    if ((s = sum_round(x, n, {{g->U, g->s, g->V, g->r, g->ld, 1.0}}, x.G, x.ldp)) != LR_OK) return s;
    x.has_g = x.G.r > 0;
  }
  if (x.has_g) {
    double ra = 0.0, rb = 0.0;
    if ((s = kernel_coeffs(x, x.R, 1.0, &ra, &rb)) != LR_OK) return s;
    if ((s = kernel_coeffs(x, x.G, 1.0, &ga, &gb)) != LR_OK) return s;
    if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.G.U, x.G.s, x.G.V, x.G.r, x.ldp, -1.0},
                              {x.E, nullptr, x.E, 1, x.ldp, ga - ra}, {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, gb - rb}},
                       x.T, x.ldp)) != LR_OK)
      return s;
    std::swap(x.R, x.T);
  }
  double rr = 0.0;
  if ((s = norm2_of(x, x.R, &rr)) != LR_OK) return s;
  const double nr0 = std::sqrt(rr);
  if (history) history[0] = nr0 > 0.0 ? 1.0 : 0.0;
  x.P.r = 0;
  if (p->r > 0 && nr0 > 0.0) {
    // Resume from the pressure given in p (a saved iterate): copied in with
    // its kernel modes removed; CG restarts from r = rhs - S p (GMRES forms
    // that residual itself).
    LR_CUDA(h, cudaMemcpy2DAsync(x.T.U, sizeof(double) * x.ldp, p->U, sizeof(double) * p->ld, sizeof(double) * n,
                                 p->r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpy2DAsync(x.T.V, sizeof(double) * x.ldp, p->V, sizeof(double) * p->ld, sizeof(double) * n,
                                 p->r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpyAsync(x.T.s, p->s, sizeof(double) * p->r, cudaMemcpyDeviceToDevice, stm), "copy");
    x.T.r = p->r;
    double ka = 0.0, kb = 0.0;
    if ((s = kernel_coeffs(x, x.T, 1.0, &ka, &kb)) != LR_OK) return s;
    if ((s = sum_round(x, n, {{x.T.U, x.T.s, x.T.V, x.T.r, x.ldp, 1.0}, {x.E, nullptr, x.E, 1, x.ldp, -ka},
                              {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -kb}}, x.P, x.ldp)) != LR_OK)
      return s;
    if (!x.gmres && x.P.r > 0) {
      if ((s = schur_product(x, x.P, x.Q, 0.1 * x.eps)) != LR_OK) return s;
      double qa = 0.0, qb = 0.0;
      if ((s = kernel_coeffs(x, x.R, 1.0, &ka, &kb)) != LR_OK) return s;
      if ((s = kernel_coeffs(x, x.Q, -1.0, &qa, &qb)) != LR_OK) return s;
      if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.Q.U, x.Q.s, x.Q.V, x.Q.r, x.ldp, -1.0},
                                {x.E, nullptr, x.E, 1, x.ldp, -(ka + qa)},
                                {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -(kb + qb)}},
                         x.T, x.ldp, kCgFloor * x.eps * nr0)) != LR_OK)
        return s;
      std::swap(x.R, x.T);
      if ((s = norm2_of(x, x.R, &rr)) != LR_OK) return s;
      if (history) history[0] = std::sqrt(rr) / nr0;
    }
  }
  int it = 0;
  if (x.gmres && nr0 > 0.0) {
    double res = 0.0;
    if ((s = stokes_gmres(x, tol, maxit, nr0, &it, &res, history)) != LR_OK) return s;
    rr = res * res;
  }
  if (!x.gmres && (s = copy_lr(x, n, x.R, x.D)) != LR_OK) return s;
  while (!x.gmres && it < maxit && nr0 > 0.0 && std::sqrt(rr) > tol * nr0 && x.D.r > 0) {
    // q = (B^T A^-1 B) d
    {
      VelocityPrecision vp(x, o.eps);
      if ((s = grad_solve(x, x.D, &rx, &ry)) != LR_OK) return s;
    }
    // q enters r - alpha q with alpha = O(1) (the Schur spectrum lies in
    // (0, 1]): rounded to a tenth of the residual's absolute level
    if ((s = div_round(x, rx, ry, x.Q, 0.1 * kCgFloor * x.eps * nr0)) != LR_OK) return s;
    double dq = 0.0;
    if ((s = inner(x, n, x.D, x.Q, &dq)) != LR_OK) return s;
    if (!(dq > 0.0)) break;  // d in the kernel (round-off): nothing left to gain
    const double alpha = rr / dq;
    // p <- p + alpha d, r <- r - alpha q, d <- r + beta d (each rounded at eps)
    if ((s = sum_round(x, n, {{x.P.U, x.P.s, x.P.V, x.P.r, x.ldp, 1.0}, {x.D.U, x.D.s, x.D.V, x.D.r, x.ldp, alpha}},
                       x.T, x.ldp)) != LR_OK) return s;
    std::swap(x.P, x.T);
    // The residual and the direction shrink by orders of magnitude while
    // their terms do not: they are rounded to the absolute level
    // kCgFloor eps ||r0|| (relative rounding would keep ever more columns of
    // cancellation noise; the floor sits well below the stopping level
    // tol_div ||r0|| for the workloads' tol_div = 10 eps, so that the
    // truncations do not slow CG down near the end).
    // The new residual also loses its components along the pressure's kernel
    // modes (round-off of the truncations would otherwise accumulate there
    // and stall CG): r - alpha q - a 1 1^T - b c c^T.
    double ka = 0.0, kb = 0.0;
    if ((s = kernel_coeffs(x, x.R, 1.0, &ka, &kb)) != LR_OK) return s;
    {
      double qa = 0.0, qb = 0.0;
      if ((s = kernel_coeffs(x, x.Q, -alpha, &qa, &qb)) != LR_OK) return s;
      ka += qa;
      kb += qb;
    }
    if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.Q.U, x.Q.s, x.Q.V, x.Q.r, x.ldp, -alpha},
                              {x.E, nullptr, x.E, 1, x.ldp, -ka}, {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -kb}},
                       x.T, x.ldp, kCgFloor * x.eps * nr0)) != LR_OK) return s;
    std::swap(x.R, x.T);
    double rr_new = 0.0;
    if ((s = norm2_of(x, x.R, &rr_new)) != LR_OK) return s;
    const double beta = rr_new / rr;
    if ((s = sum_round(x, n, {{x.R.U, x.R.s, x.R.V, x.R.r, x.ldp, 1.0}, {x.D.U, x.D.s, x.D.V, x.D.r, x.ldp, beta}},
                       x.T, x.ldp, kCgFloor * x.eps * nr0)) != LR_OK) return s;
    std::swap(x.D, x.T);
    rr = rr_new;
    ++it;
    if (history) history[it] = std::sqrt(rr) / nr0;
  }
  // Project the pressure's kernel modes (constant, checkerboard) out of p.
  if (x.P.r > 0) {
    double a = 0.0, b2 = 0.0;
    if ((s = kernel_coeffs(x, x.P, 1.0, &a, &b2)) != LR_OK) return s;
    if ((s = sum_round(x, n, {{x.P.U, x.P.s, x.P.V, x.P.r, x.ldp, 1.0}, {x.E, nullptr, x.E, 1, x.ldp, -a},
                              {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, -b2}}, x.T, x.ldp)) != LR_OK) return s;
    std::swap(x.P, x.T);
  }
  // Velocity u = A^-1 (f - B p), the right-hand sides rounded first (f and
  // B p cancel in part) with their weights folded into U.
  lr_mat rhs[2];
  const int m = n - 1;
  const double c = n / 4.0;
  for (int k = 0; k < 2; ++k) {
    double* GU = x.b.FU;  // gradient factors of this component (scratch)
    double* GV = x.b.FV;
    LR_CUDA(h, launch_gh(k == 0 ? OP_G : OP_H, n, x.P.U, x.ldp, x.P.r, x.P.s, c, GU, x.ldv, stm), "grad");
    LR_CUDA(h, launch_gh(k == 0 ? OP_H : OP_G, n, x.P.V, x.ldp, x.P.r, nullptr, 1.0, GV, x.ldv, stm), "grad");
    LrDev out{x.RU[k], x.T.s, x.RV[k], 0};
    if ((s = sum_round(x, m, {{f[k].U, nullptr, f[k].V, f[k].r, f[k].ld, 1.0}, {GU, nullptr, GV, x.P.r, x.ldv, -1.0}},
                       out, x.ldv)) != LR_OK) return s;
    rhs[k] = {m, m, out.r, out.r, x.ldv, x.RU[k], nullptr, x.RV[k]};
    if (out.r == 0) {  // f = B p: a zero column, whose solve is rank 0
      LR_CUDA(h, cudaMemsetAsync(x.RU[k], 0, sizeof(double) * m, stm), "zero");
      LR_CUDA(h, cudaMemsetAsync(x.RV[k], 0, sizeof(double) * m, stm), "zero");
      rhs[k].r = rhs[k].rmax = 1;
    } else {
      LR_CUDA(h, launch_fold_weights(m, KMAX, &x.b.st->rank, x.RU[k], x.ldv, x.T.s, false, stm), "fold");
    }
  }
  // the solutions go straight into the caller's buffers
  std::vector<Plan*> plans(2, x.plan);
  {
    VelocityPrecision vp(x, o.eps);
    lr_options of = x.oin;
    s = x.oin.prec == LR_MIXED ? solve2d_batched<float>(h, 2, rhs, u, of, plans, nullptr, false)
                               : solve2d_batched<double>(h, 2, rhs, u, of, plans, nullptr, false);
  }
  if (s != LR_OK && s != LR_ENOCONV) return s;
  // divergence of the final velocity, relative to ||B^T A^-1 f||
  for (int k = 0; k < 2; ++k) {
    LR_CUDA(h, cudaMemcpy2DAsync(x.WU[k], sizeof(double) * x.ldv, u[k].U, sizeof(double) * u[k].ld,
                                 sizeof(double) * m, u[k].r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpy2DAsync(x.WV[k], sizeof(double) * x.ldv, u[k].V, sizeof(double) * u[k].ld,
                                 sizeof(double) * m, u[k].r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpyAsync(x.Ws[k], u[k].s, sizeof(double) * u[k].r, cudaMemcpyDeviceToDevice, stm), "copy");
  }
  if ((s = div_round(x, u[0].r, u[1].r, x.T)) != LR_OK) return s;
  if (x.has_g) {  // B^T u - (g without its kernel components)
    if ((s = sum_round(x, n, {{x.T.U, x.T.s, x.T.V, x.T.r, x.ldp, 1.0}, {x.G.U, x.G.s, x.G.V, x.G.r, x.ldp, -1.0},
                              {x.E, nullptr, x.E, 1, x.ldp, ga}, {x.E + x.ldp, nullptr, x.E + x.ldp, 1, x.ldp, gb}},
                       x.Q, x.ldp)) != LR_OK)
      return s;
    std::swap(x.T, x.Q);
  }
  double dv = 0.0;
  if ((s = norm2_of(x, x.T, &dv)) != LR_OK) return s;
  // pressure out
  if (x.P.r > p->rmax) return fail(h, LR_ENOCONV, "pressure rank exceeds p->rmax");
  if (x.P.r > 0) {
    LR_CUDA(h, cudaMemcpy2DAsync(p->U, sizeof(double) * p->ld, x.P.U, sizeof(double) * x.ldp, sizeof(double) * n,
                                 x.P.r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpy2DAsync(p->V, sizeof(double) * p->ld, x.P.V, sizeof(double) * x.ldp, sizeof(double) * n,
                                 x.P.r, cudaMemcpyDeviceToDevice, stm), "copy");
    LR_CUDA(h, cudaMemcpyAsync(p->s, x.P.s, sizeof(double) * x.P.r, cudaMemcpyDeviceToDevice, stm), "copy");
  }
  LR_CUDA(h, cudaStreamSynchronize(stm), "Stokes");
  p->r = x.P.r;
  if (iters) *iters = it;
  const double res = nr0 > 0.0 ? std::sqrt(dv) / nr0 : 0.0;
  if (resid) *resid = res;
  h->info = lr_info{};
  h->info.launches = x.launches;
  h->info.rank = x.P.r;
  h->info.refine_rounds = x.escalations;  // reused: velocity solves escalated to float64
  if (!(std::sqrt(rr) <= tol * nr0) && nr0 > 0.0)
    return fail(h, LR_ENOCONV, "Uzawa did not reach tol_div within maxit");
  if (x.cut) return fail(h, LR_ENOCONV, "a low-rank sum needed more than 64 columns; columns were dropped");
  return LR_OK;
}

}  // namespace

extern "C" {

void lr_options_default(lr_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->prec = LR_MIXED;
  o->op = LR_OP_5PT;
  o->eps = 1e-6;
  o->rmax = KMAX;
  o->aca_tol_factor = 1.0;
  o->probes = 16;
  o->seed = 0;
  o->flags = 0;
  o->cluster_size = 0;
  o->refine = 0;
}

const char* lr_status_string(lr_status s) {
  switch (s) {
    case LR_OK: return "LR_OK";
    case LR_EINVAL: return "LR_EINVAL";
    case LR_ENOMEM: return "LR_ENOMEM";
    case LR_ENOCONV: return "LR_ENOCONV";
    case LR_ETIMEOUT: return "LR_ETIMEOUT";
    case LR_ECUDA: return "LR_ECUDA";
    case LR_ENONFINITE: return "LR_ENONFINITE";
  }
  return "unknown";
}

lr_status lr_create(lr_handle* out, void* stream) {
  if (!out) return LR_EINVAL;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LR_ECUDA; }
  lr_handle h = new lr_handle_s();
  h->stream = static_cast<cudaStream_t>(stream);
  h->device = dev;
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LR_ECUDA;
  }
  if (cudaMallocHost(&h->h_state, sizeof(SolveState)) != cudaSuccess ||
      cudaMallocHost(&h->h_piv, sizeof(int) * 2 * KMAX) != cudaSuccess ||
      cudaMallocHost(&h->h_w, sizeof(double) * 2 * KMAX) != cudaSuccess) {
    cudaGetLastError();
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->h_piv) cudaFreeHost(h->h_piv);
    delete h;
    return LR_ENOMEM;
  }
  std::memset(h->h_state, 0, sizeof(SolveState));
  std::memset(h->h_piv, 0, sizeof(int) * 2 * KMAX);
  *out = h;
  return LR_OK;
}

lr_status lr_set_workspace_limit(lr_handle h, size_t bytes) {
  if (!h) return LR_EINVAL;
  h->ws_limit = bytes;
  return LR_OK;
}

lr_status lr_set_stream(lr_handle h, void* stream) {
  if (!h) return LR_EINVAL;
  h->stream = static_cast<cudaStream_t>(stream);
  return LR_OK;
}

lr_status lr_destroy(lr_handle h) {
  if (!h) return LR_EINVAL;
  cudaStreamSynchronize(h->stream);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->graph_desc) cudaFree(kv.second);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (void* t : h->tw4096)
    if (t) cudaFree(t);
  if (h->bdesc) cudaFree(h->bdesc);
  if (h->h_bdesc) cudaFreeHost(h->h_bdesc);
  if (h->bdesc_ev) cudaEventDestroy(h->bdesc_ev);
  for (int i = 0; i < 32; ++i) {
    if (h->bstreams[i]) cudaStreamDestroy(h->bstreams[i]);
    if (h->bjoin[i]) cudaEventDestroy(h->bjoin[i]);
  }
  if (h->bfork) cudaEventDestroy(h->bfork);
  if (h->h_bstate) cudaFreeHost(h->h_bstate);
  h->plans.clear();
  if (h->ws) cudaFree(h->ws);
  if (h->ws2) cudaFree(h->ws2);
  if (h->ws3) cudaFree(h->ws3);
  if (h->ws4) cudaFree(h->ws4);
  if (h->ws5) cudaFree(h->ws5);
  if (h->h_big) cudaFreeHost(h->h_big);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_piv) cudaFreeHost(h->h_piv);
  if (h->h_w) cudaFreeHost(h->h_w);
  delete h;
  return LR_OK;
}

const char* lr_last_error(lr_handle h) { return h ? h->err.c_str() : "null handle"; }

lr_status lr_dst1(lr_handle h, int m, int ncols, const double* in, int ld_in, double* out, int ld_out,
                  lr_precision prec) {
  if (!h) return LR_EINVAL;
  if (m < 1 || ncols < 0 || ld_in < m || ld_out < m) return fail(h, LR_EINVAL, "lr_dst1: bad sizes");
  if (ncols == 0) return LR_OK;
  if (!in || !out || !aligned16(in) || !aligned16(out)) return fail(h, LR_EINVAL, "lr_dst1: null or unaligned pointer");
  if (prec != LR_FP64 && prec != LR_MIXED) return fail(h, LR_EINVAL, "lr_dst1: unknown precision");
  Plan* plan = nullptr;
  lr_status s = get_plan(h, m, &plan);
  if (s != LR_OK) return s;
  const size_t M = (size_t)1 << plan->logM;
  const size_t esz = prec == LR_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
  s = ensure_ws(h, M > (size_t)kSmallM ? M * ncols * esz : 256);
  if (s != LR_OK) return s;
  ColumnSet cs;
  cs.in[0] = in; cs.out[0] = out; cs.ld_in[0] = ld_in; cs.ld_out[0] = ld_out; cs.ncol[0] = ncols;
  cudaError_t e = prec == LR_FP64
                      ? launch_dst<double>(*plan, cs, IoType::F64, IoType::F64, h->ws, h->num_sms, h->stream)
                      : launch_dst<float>(*plan, cs, IoType::F64, IoType::F64, h->ws, h->num_sms, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "lr_dst1");
  LR_CUDA(h, cudaStreamSynchronize(h->stream), "lr_dst1");
  return LR_OK;
}

lr_status lr_poisson2d_full(lr_handle h, int m, const double* F, int ldf, double* X, int ldx,
                            const lr_options* opt) {
  NvtxRange nvtx_range("lr_poisson2d_full");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  if (o.prec != LR_FP64 && o.prec != LR_MIXED) return fail(h, LR_EINVAL, "unknown precision");
  if (o.op != LR_OP_5PT && o.op != LR_OP_SEMISTAGGERED) return fail(h, LR_EINVAL, "unknown operator");
  if (m < 1 || m > 65536) return fail(h, LR_EINVAL, "m must be in [1, 65536]");
  if (ldf < m || ldx < m) return fail(h, LR_EINVAL, "leading dimension smaller than m");
  if (!F || !X || !aligned16(F) || !aligned16(X)) return fail(h, LR_EINVAL, "null or unaligned pointer");
  if (F == X) return fail(h, LR_EINVAL, "X may not alias F");
  Plan* plan = nullptr;
  lr_status s = get_plan(h, m, &plan);
  if (s != LR_OK) return s;
  return o.prec == LR_MIXED ? solve2d_full<float>(h, m, F, ldf, X, ldx, o, plan)
                            : solve2d_full<double>(h, m, F, ldf, X, ldx, o, plan);
}

lr_status lr_poisson2d(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options* opt) {
  NvtxRange nvtx_range("lr_poisson2d");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if ((s = check_problem(h, rhs, sol)) != LR_OK) return s;
  const int m = rhs->n1;
  Plan* plan = nullptr;
  s = get_plan(h, m, &plan);
  if (s != LR_OK) return s;
  h->info = lr_info{};
  if (o.cluster_size == 0) {  // autotuned configuration of this order, if any
    auto it = h->tuned_cs.find(std::make_tuple(m, (int)o.prec, (int)o.op));
    if (it != h->tuned_cs.end()) o.cluster_size = it->second;
  }
  int rounds = o.refine;
  if (rounds == 0) rounds = o.eps < 1e-7 ? 6 : 0;
  if (o.prec == LR_MIXED && rounds > 0)
    s = solve2d_refined(h, rhs, sol, o, plan, rounds);
  else
    s = o.prec == LR_MIXED ? solve2d<float>(h, rhs, sol, o, plan) : solve2d<double>(h, rhs, sol, o, plan);
  h->info.status = s;
  return s;
}

lr_status lr_poisson2d_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options* opt,
                               lr_status* per_problem) {
  NvtxRange nvtx_range("lr_poisson2d_batched");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (batch < 0 || (batch > 0 && (!rhs || !sol))) return fail(h, LR_EINVAL, "bad batch arguments");
  if (batch == 0) return LR_OK;
  if ((o.flags & LR_FLAG_TIMING) &&
      ((o.flags & LR_FLAG_BATCH_STREAMS) || !batch_phased_fits(batch, rhs, o.prec == LR_MIXED)))
    return fail(h, LR_EINVAL, "LR_FLAG_TIMING needs the phase-batched form");
  std::vector<Plan*> plans(batch);
  for (int i = 0; i < batch; ++i) {
    if ((s = check_problem(h, &rhs[i], &sol[i])) != LR_OK) {
      if (per_problem) per_problem[i] = s;
      return fail(h, s, "problem " + std::to_string(i) + ": " + h->err);
    }
    if ((s = get_plan(h, rhs[i].n1, &plans[i])) != LR_OK) return s;
  }
  h->info = lr_info{};
  h->timed = false;
  h->last_batch = 0;
  s = o.prec == LR_MIXED ? solve2d_batched<float>(h, batch, rhs, sol, o, plans, per_problem)
                         : solve2d_batched<double>(h, batch, rhs, sol, o, plans, per_problem);
  if (s == LR_OK || s == LR_ENOCONV || s == LR_ENONFINITE) h->last_batch = batch;
  h->info.status = s;
  return s;
}

lr_status lr_batched_status(lr_handle h, int batch, lr_mat* sol, lr_status* per_problem) {
  if (!h) return LR_EINVAL;
  if (batch < 0 || (batch > 0 && !sol)) return fail(h, LR_EINVAL, "bad batch arguments");
  if (batch > h->last_batch)
    return fail(h, LR_EINVAL, "batch exceeds the last batched call on this handle");
  return collect_batch(h, batch, sol, per_problem);
}

// Autotuning: time candidate launch shapes on the caller's problem (CUDA
// events on the handle's stream, median of reps after a warm-up).
lr_status lr_stokes_uzawa(lr_handle h, int d, int n, const lr_mat* f, const lr_mat* g, lr_mat* u, lr_mat* p,
                          double tol_div, int maxit, const lr_options* opt, int* iters, double* resid,
                          double* history) {
  NvtxRange nvtx_range("lr_stokes_uzawa");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (d != 2) return fail(h, LR_EINVAL, "lr_stokes_uzawa: only d = 2 is built");
  if (g && (g->n1 != n || g->n2 != n || g->r < 0 || g->r > KMAX || g->ld < n || !g->U || !g->V ||
            !aligned16(g->U) || !aligned16(g->V) || (g->s && !aligned16(g->s))))
    return fail(h, LR_EINVAL, "lr_stokes_uzawa: g must be NULL or n x n of rank 0..64 with aligned U, V");
  if (n < 3 || n > 32768) return fail(h, LR_EINVAL, "lr_stokes_uzawa: n must be in [3, 32768]");
  if (!f || !u || !p) return fail(h, LR_EINVAL, "lr_stokes_uzawa: null f, u or p");
  if (!(tol_div > 0.0) || tol_div >= 1.0 || maxit < 1) return fail(h, LR_EINVAL, "lr_stokes_uzawa: bad tol_div or maxit");
  const int m = n - 1;
  for (int k = 0; k < 2; ++k) {
    if (f[k].n1 != m || f[k].n2 != m || u[k].n1 != m || u[k].n2 != m)
      return fail(h, LR_EINVAL, "lr_stokes_uzawa: f and u components must be (n-1) x (n-1)");
    if ((s = check_problem(h, &f[k], &u[k])) != LR_OK) return s;
  }
  if (p->n1 != n || p->n2 != n || p->ld < n || p->rmax < 1 || !p->U || !p->V || !p->s ||
      !aligned16(p->U) || !aligned16(p->V) || !aligned16(p->s))
    return fail(h, LR_EINVAL, "lr_stokes_uzawa: p must be n x n with U, s, V set and aligned");
  if (p->r < 0 || p->r > std::min(p->rmax, KMAX))
    return fail(h, LR_EINVAL, "lr_stokes_uzawa: p->r (the initial guess's rank, 0 for none) must be in [0, min(p->rmax, 64)]");
  return stokes_uzawa(h, n, f, g, u, p, tol_div, maxit, o, iters, resid, history);
}

lr_status lr_poisson3d_tucker(lr_handle h, const lr_tucker* rhs, lr_tucker* sol, const lr_options* opt) {
  NvtxRange nvtx_range("lr_poisson3d_tucker");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (o.prec != LR_FP64 && o.prec != LR_MIXED) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: unknown precision");
  if (o.prec == LR_MIXED && !(o.eps >= 1e-7))
    return fail(h, LR_EINVAL, "lr_poisson3d_tucker: LR_MIXED needs eps >= 1e-7 (float32 transforms and cores)");
  if (o.op != LR_OP_5PT) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: the 7-point operator (LR_OP_5PT kind) only");
  if (!rhs || !sol || !rhs->G || !sol->G) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: null rhs, sol or core");
  for (int k = 0; k < 3; ++k) {
    if (rhs->n[k] < 1 || rhs->n[k] > 16384) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: n[k] must be in [1, 16384]");
    if (rhs->r[k] < 1 || rhs->r[k] > KMAX) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: r[k] must be in [1, 64]");
    if (rhs->ld[k] < rhs->n[k] || sol->ld[k] < rhs->n[k]) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: ld[k] < n[k]");
    if (sol->n[k] != rhs->n[k]) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: sol->n must equal rhs->n");
    if (sol->rmax[k] < 1 || sol->rmax[k] > KMAX) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: sol->rmax[k] must be in [1, 64]");
    if (!rhs->U[k] || !sol->U[k] || !aligned16(rhs->U[k]) || !aligned16(sol->U[k]) || (rhs->ld[k] & 1) ||
        (sol->ld[k] & 1))
      return fail(h, LR_EINVAL, "lr_poisson3d_tucker: factors must be 16-byte aligned with even ld");
  }
  if (!aligned16(rhs->G) || !aligned16(sol->G)) return fail(h, LR_EINVAL, "lr_poisson3d_tucker: cores must be 16-byte aligned");
  return solve3d_tucker(h, rhs, sol, o);
}

lr_status lr_poisson2d_expsum(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options* opt, int* nterms) {
  NvtxRange nvtx_range("lr_poisson2d_expsum");
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (o.op != LR_OP_5PT) return fail(h, LR_EINVAL, "exp-sum: the 5-point kind only (the other symbol does not split)");
  if (!(o.eps >= 1e-12)) return fail(h, LR_EINVAL, "exp-sum: eps must be >= 1e-12");
  if ((s = check_problem(h, rhs, sol)) != LR_OK) return s;
  Plan* plan = nullptr;
  if ((s = get_plan(h, rhs->n1, &plan)) != LR_OK) return s;
  return solve2d_expsum(h, rhs, sol, o, plan, nterms);
}

lr_status lr_autotune(lr_handle h, const lr_mat* rhs, const lr_options* opt, int reps, lr_tune* out) {
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (!rhs) return fail(h, LR_EINVAL, "null rhs");
  if (reps < 1 || reps > 100) return fail(h, LR_EINVAL, "reps must be in [1, 100]");
  const int m = rhs->n1;
  const int ld = m + (m & 1);
  double* buf = nullptr;
  if (m < 1 || m > 131072) return fail(h, LR_EINVAL, "m must be in [1, 131072]");
  if (cudaMalloc(&buf, sizeof(double) * ((size_t)2 * ld * KMAX + KMAX)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, LR_ENOMEM, "autotune scratch");
  }
  struct Free { double* p; ~Free() { cudaFree(p); } } guard{buf};
  lr_mat sol = {m, m, 0, KMAX, ld, buf, buf + (size_t)2 * ld * KMAX, buf + (size_t)ld * KMAX};
  if ((s = check_problem(h, rhs, &sol)) != LR_OK) return s;
  Plan* plan = nullptr;
  if ((s = get_plan(h, m, &plan)) != LR_OK) return s;
  if ((s = ensure_events(h)) != LR_OK) return s;
  o.flags = LR_FLAG_TIMING;
  o.refine = -1;
  const int pi = o.prec == LR_MIXED ? 1 : 0;
  int ncand = 0;
  auto timed = [&](int cs, int tile, double* ms, int* used) -> lr_status {
    // tile -1: the cluster transform; otherwise the four-step tile (0: heuristic)
    plan->use_cluster[pi] = tile < 0 ? 1 : 0;
    plan->log_tile[pi] = tile < 0 ? 0 : tile;
    o.cluster_size = cs;
    std::vector<double> t;
    for (int i = 0; i <= reps; ++i) {
      const lr_status st = o.prec == LR_MIXED ? solve2d<float>(h, rhs, &sol, o, plan)
                                              : solve2d<double>(h, rhs, &sol, o, plan);
      if (st != LR_OK && st != LR_ENOCONV) return st;
      float e = 0.f;
      LR_CUDA(h, cudaEventElapsedTime(&e, h->ev[0], h->ev[LR_NUM_PHASES]), "event time");
      if (i > 0) t.push_back(e);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    *used = h->last_cs;
    ++ncand;
    return LR_OK;
  };
  double ms_def = 0.0, ms = 0.0;
  int used = 0, best_cs = 0, best_tile = 0;
  if ((s = timed(0, 0, &ms_def, &best_cs)) != LR_OK) return s;
  double best = ms_def;
  const int logM = plan->logM;
  if (((size_t)1 << logM) > (size_t)kSmallM) {  // four-step transform: tile 2^10 .. 2^12
    const int logMin = std::max((logM + 1) / 2, 10);
    for (int t = logMin; t <= 12; ++t) {
      if ((s = timed(0, t, &ms, &used)) != LR_OK) return s;
      if (ms < best) { best = ms; best_tile = t; best_cs = used; }
    }
    if (plan->logN2cl) {
      if ((s = timed(0, -1, &ms, &used)) != LR_OK) return s;
      if (ms < best) { best = ms; best_tile = -1; best_cs = used; }
    }
  }
  const int cs_min = (m + 8191) / 8192;
  const int cs_max = std::min(16, std::max(1, (m + 127) / 128));
  for (int cs : {1, 2, 4, 8, 12, 16}) {
    if (cs < cs_min || cs > cs_max) continue;
    if ((s = timed(cs, best_tile, &ms, &used)) != LR_OK) return s;
    if (ms < best) { best = ms; best_cs = used; }
  }
  plan->use_cluster[pi] = best_tile < 0 ? 1 : 0;
  plan->log_tile[pi] = best_tile < 0 ? 0 : best_tile;
  h->tuned_cs[std::make_tuple(m, (int)o.prec, (int)o.op)] = best_cs;
  h->timed = false;
  ++h->ws_gen;  // graphs captured before tuning bake in the untuned shapes
  if (out) {
    out->cluster_size = best_cs;
    out->log_tile = best_tile < 0 ? 0 : best_tile;
    out->transform = best_tile < 0 ? 1 : 0;
    out->batch_indices_per_cta = h->batch_ipc[pi];
    out->candidates = ncand;
    out->ms_best = best;
    out->ms_default = ms_def;
  }
  return LR_OK;
}

lr_status lr_autotune_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options* opt,
                              int reps, lr_tune* out) {
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (batch < 1 || !rhs || !sol) return fail(h, LR_EINVAL, "bad batch arguments");
  if (reps < 1 || reps > 100) return fail(h, LR_EINVAL, "reps must be in [1, 100]");
  std::vector<Plan*> plans(batch);
  for (int i = 0; i < batch; ++i) {
    if ((s = check_problem(h, &rhs[i], &sol[i])) != LR_OK) return s;
    if ((s = get_plan(h, rhs[i].n1, &plans[i])) != LR_OK) return s;
  }
  if ((s = ensure_events(h)) != LR_OK) return s;
  const bool streams = (o.flags & LR_FLAG_BATCH_STREAMS) != 0 ||
                       !batch_phased_fits(batch, rhs, o.prec == LR_MIXED);
  o.flags &= LR_FLAG_BATCH_STREAMS;
  o.cluster_size = 0;
  const int pi = o.prec == LR_MIXED ? 1 : 0;
  // the stream form tunes the indices per cross CTA of its per-problem
  // clusters; the phase-batched form those of its batched cross (1, 2 or 4
  // CTAs per problem)
  int& knob = streams ? h->batch_ipc[pi] : h->cross_rows[pi];
  const int before = knob;
  std::vector<int> cands = streams ? std::vector<int>{2048, 1024, 4096, 8192}
                                   : std::vector<int>{4096, 2048, 8192, 16384};
  if (!streams)
    cands.erase(std::remove_if(cands.begin(), cands.end(),
                               [&](int c2) { return c2 > batch_cross_max_rows(o.prec == LR_MIXED); }),
                cands.end());
  double best = 0.0, ms_def = 0.0;
  int best_ipc = before, ncand = 0;
  for (int ipc : cands) {  // the default first
    knob = ipc;
    std::vector<double> t;
    for (int i = 0; i <= reps; ++i) {
      LR_CUDA(h, cudaEventRecord(h->ev[0], h->stream), "event");
      const lr_status st = o.prec == LR_MIXED ? solve2d_batched<float>(h, batch, rhs, sol, o, plans, nullptr)
                                              : solve2d_batched<double>(h, batch, rhs, sol, o, plans, nullptr);
      if (st != LR_OK && st != LR_ENOCONV) { knob = before; return st; }
      LR_CUDA(h, cudaEventRecord(h->ev[1], h->stream), "event");
      LR_CUDA(h, cudaEventSynchronize(h->ev[1]), "event");
      float e = 0.f;
      LR_CUDA(h, cudaEventElapsedTime(&e, h->ev[0], h->ev[1]), "event time");
      if (i > 0) t.push_back(e);
    }
    std::sort(t.begin(), t.end());
    const double ms = t[t.size() / 2];
    if (ncand == 0) ms_def = ms;
    ++ncand;
    if (ncand == 1 || ms < best) { best = ms; best_ipc = ipc; }
  }
  knob = best_ipc;
  h->timed = false;
  ++h->ws_gen;  // graphs captured before tuning bake in the untuned shapes
  if (out) {
    auto it = h->tuned_cs.find(std::make_tuple(rhs[0].n1, (int)o.prec, (int)o.op));
    out->cluster_size = it != h->tuned_cs.end() ? it->second : 0;
    Plan* p0 = plans[0];
    out->log_tile = p0->log_tile[pi];
    out->transform = p0->use_cluster[pi];
    out->batch_indices_per_cta = best_ipc;
    out->candidates = ncand;
    out->ms_best = best;
    out->ms_default = ms_def;
  }
  return LR_OK;
}

lr_status lr_maxvol(lr_handle h, const double* C, int m, int k, int ldc, double delta, int maxswaps,
                    int* rows, int* nswaps, double* bmax) {
  NvtxRange nvtx_range("lr_maxvol");
  if (!h) return LR_EINVAL;
  if (!C || !rows) return fail(h, LR_EINVAL, "C and rows must be set");
  if (k < 1 || k > MV_KMAX || m < k || ldc < m) return fail(h, LR_EINVAL, "need 1 <= k <= min(64, m), ldc >= m");
  if (!(delta >= 0.0) || !(delta < 1e300)) return fail(h, LR_EINVAL, "delta must be finite and >= 0");
  if (maxswaps < 0) return fail(h, LR_EINVAL, "maxswaps must be >= 0");
  for (int j = 0; j < k; ++j) {
    if (rows[j] < 0 || rows[j] >= m) return fail(h, LR_EINVAL, "rows must lie in [0, m)");
    for (int l = 0; l < j; ++l)
      if (rows[l] == rows[j]) return fail(h, LR_EINVAL, "rows must be distinct");
  }
  const int grid = maxvol_grid(m, h->num_sms);
  const int ldb = round_up(m, 32);
  auto layout = [&](Carve& cv, MvArgs& a) {
    a.B = cv.take<double>(sizeof(double) * (size_t)ldb * k);
    a.Ainv = cv.take<double>(sizeof(double) * MV_KMAX * MV_KMAX);
    a.row = cv.take<double>(sizeof(double) * MV_KMAX);
    a.pabs = cv.take<double>(sizeof(double) * grid);
    a.pidx = cv.take<long long>(sizeof(long long) * grid);
    a.rows = cv.take<int>(sizeof(int) * MV_KMAX);
    a.st = cv.take<MvState>(sizeof(MvState));
  };
  MvArgs a{};
  Carve c;
  layout(c, a);
  lr_status s = ensure_ws(h, c.off);
  if (s != LR_OK) return s;
  Carve c2;
  c2.base = static_cast<char*>(h->ws);
  layout(c2, a);
  a.C = C;
  a.ldc = ldc;
  a.m = m;
  a.k = k;
  a.delta = delta;
  a.maxswaps = maxswaps;
  a.ldb = ldb;
  a.grid = grid;
  cudaStream_t stm = h->stream;
  MvState hs{};
  LR_CUDA(h, cudaMemsetAsync(a.st, 0, sizeof(MvState), stm), "maxvol state");
  LR_CUDA(h, cudaMemcpyAsync(a.rows, rows, sizeof(int) * k, cudaMemcpyHostToDevice, stm), "maxvol rows in");
  LR_CUDA(h, launch_maxvol_start(a, stm), "maxvol start");
  // Swaps in groups of 32, the record read between groups; at most maxswaps
  // swap launches in all (the decision after the last one stops).
  for (int launched = 0;;) {
    LR_CUDA(h, cudaMemcpyAsync(&hs, a.st, sizeof(MvState), cudaMemcpyDeviceToHost, stm), "maxvol state out");
    LR_CUDA(h, cudaStreamSynchronize(stm), "maxvol");
    if (hs.done || launched >= maxswaps) break;
    const int g = maxswaps - launched < 32 ? maxswaps - launched : 32;
    for (int q = 0; q < g; ++q) LR_CUDA(h, launch_maxvol_swap(a, stm), "maxvol swap");
    launched += g;
  }
  LR_CUDA(h, cudaMemcpyAsync(rows, a.rows, sizeof(int) * k, cudaMemcpyDeviceToHost, stm), "maxvol rows out");
  LR_CUDA(h, cudaStreamSynchronize(stm), "maxvol rows");
  if (nswaps) *nswaps = hs.nswaps;
  if (bmax) *bmax = hs.bmax;
  if (hs.status & 1) return fail(h, LR_EINVAL, "C[rows, :] is singular or not finite");
  if (hs.status & 2) return fail(h, LR_ENONFINITE, "non-finite coefficient in C C[rows, :]^-1");
  if (!hs.done || hs.bmax > 1.0 + delta) return fail(h, LR_ENOCONV, "maxswaps swaps made, max |B| > 1 + delta");
  return LR_OK;
}

lr_status lr_get_info(lr_handle h, lr_info* info, int* pivots_I, int* pivots_J, int cap) {
  if (!h || !info) return LR_EINVAL;
  const SolveState& hs = *h->h_state;
  const int cs = h->info.cluster_size;
  *info = h->info;
  info->aca_steps = hs.k;
  info->rank = hs.rank;
  info->converged = hs.converged;
  info->cut = hs.cut;
  info->probe_rounds = hs.probe_rounds;
  info->zero_rows = hs.zero_rows;
  info->norm_est = std::sqrt(hs.norm2 > 0 ? hs.norm2 : 0.0);
  info->sigma0 = hs.sigma0;
  info->cluster_size = cs;
  info->launches = h->info.launches;
  if (info->status == LR_OK && (!hs.converged || hs.cut)) info->status = LR_ENOCONV;
  const int n = hs.k < cap ? hs.k : cap;
  for (int i = 0; i < n; ++i) {
    if (pivots_I) pivots_I[i] = h->h_piv[i];
    if (pivots_J) pivots_J[i] = h->h_piv[KMAX + i];
  }
  return LR_OK;
}

lr_status lr_get_phase_times(lr_handle h, double* ms, int n) {
  if (!h || !ms || n < 0) return LR_EINVAL;
  if (!h->timed) return fail(h, LR_EINVAL, "the last solve was not run with LR_FLAG_TIMING");
  LR_CUDA(h, cudaEventSynchronize(h->ev[LR_NUM_PHASES]), "event sync");
  for (int i = 0; i < n && i < LR_NUM_PHASES; ++i) {
    float t = 0.f;
    LR_CUDA(h, cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]), "event elapsed");
    ms[i] = (double)t;
  }
  return LR_OK;
}

lr_status lr_truncate(lr_handle h, lr_mat* X, double eps, int rmax) {
  NvtxRange nvtx_range("lr_truncate");
  if (!h) return LR_EINVAL;
  if (!X) return fail(h, LR_EINVAL, "null matrix");
  if (!(eps > 0.0) || eps >= 1.0) return fail(h, LR_EINVAL, "eps must be in (0, 1)");
  const int k = X->r;
  if (k < 1 || k > KMAX || X->rmax < k) return fail(h, LR_EINVAL, "X->r must be in [1, min(64, rmax)]");
  if (X->n1 < 1 || X->n2 < 1 || X->ld < X->n1 || X->ld < X->n2) return fail(h, LR_EINVAL, "bad sizes");
  if (rmax < 1) return fail(h, LR_EINVAL, "rmax must be >= 1");
  if (!X->U || !X->V || !X->s) return fail(h, LR_EINVAL, "X->U, X->V and X->s must be set");
  if (!aligned16(X->U) || !aligned16(X->V) || !aligned16(X->s)) return fail(h, LR_EINVAL, "unaligned pointer");
  const int keep_cap = rmax < X->rmax ? rmax : X->rmax;
  const int n1 = X->n1, n2 = X->n2;
  const int nmax = n1 > n2 ? n1 : n2;
  const int ldw = round_up(nmax, 32);
  const int nblk = (nmax + 63) / 64;
  Carve c;
  auto layout = [&](Carve& cv, double** GU, double** GV, double** part, double** Tc, double** Tr, double** w,
                    double** Ut, double** Vt, SolveState** st) {
    *GU = cv.take<double>(sizeof(double) * k * k);
    *GV = cv.take<double>(sizeof(double) * k * k);
    *part = cv.take<double>(sizeof(double) * KMAX * KMAX * nblk);
    *Tc = cv.take<double>(sizeof(double) * KMAX * KMAX);
    *Tr = cv.take<double>(sizeof(double) * KMAX * KMAX);
    *w = cv.take<double>(sizeof(double) * KMAX);
    *Ut = cv.take<double>(sizeof(double) * ldw * k);
    *Vt = cv.take<double>(sizeof(double) * ldw * k);
    *st = cv.take<SolveState>(sizeof(SolveState));
  };
  double *GU, *GV, *part, *Tc, *Tr, *w, *Ut, *Vt;
  SolveState* st;
  layout(c, &GU, &GV, &part, &Tc, &Tr, &w, &Ut, &Vt, &st);
  lr_status s = ensure_ws(h, c.off);
  if (s != LR_OK) return s;
  Carve c2;
  c2.base = static_cast<char*>(h->ws);
  layout(c2, &GU, &GV, &part, &Tc, &Tr, &w, &Ut, &Vt, &st);
  cudaStream_t stm = h->stream;
  LR_CUDA(h, cudaMemsetAsync(st, 0, sizeof(SolveState), stm), "state reset");
  LR_CUDA(h, cudaMemcpyAsync(w, X->s, sizeof(double) * k, cudaMemcpyDeviceToDevice, stm), "weights");
  LR_CUDA(h, launch_gram(X->U, n1, X->ld, k, GU, k, part, h->num_sms, stm), "gram U");
  LR_CUDA(h, launch_gram(X->V, n2, X->ld, k, GV, k, part, h->num_sms, stm), "gram V");
  CoreArgs<double> co;
  co.GC = GU; co.GR = GV; co.ldg = k; co.d = w;
  co.k_dev = nullptr; co.k_host = k;
  co.eps = eps; co.rmax_out = keep_cap;
  co.Tc = Tc; co.Tr = Tr; co.s_out = X->s; co.st = st;
  LR_CUDA(h, launch_core<double>(co, false, stm), "rounding core");
  LR_CUDA(h, (launch_rotate<double, double>(X->U, X->ld, n1, nullptr, k, Tc, false, &st->rank, Ut, ldw, stm)),
          "rotation U");
  LR_CUDA(h, (launch_rotate<double, double>(X->V, X->ld, n2, nullptr, k, Tr, false, &st->rank, Vt, ldw, stm)),
          "rotation V");
  LR_CUDA(h, cudaMemcpyAsync(h->h_state, st, sizeof(SolveState), cudaMemcpyDeviceToHost, stm), "state copy");
  LR_CUDA(h, cudaStreamSynchronize(stm), "lr_truncate");
  const int R = h->h_state->rank;
  if (R > 0) {
    LR_CUDA(h, cudaMemcpy2DAsync(X->U, sizeof(double) * X->ld, Ut, sizeof(double) * ldw, sizeof(double) * n1, R,
                                 cudaMemcpyDeviceToDevice, stm), "copy U");
    LR_CUDA(h, cudaMemcpy2DAsync(X->V, sizeof(double) * X->ld, Vt, sizeof(double) * ldw, sizeof(double) * n2, R,
                                 cudaMemcpyDeviceToDevice, stm), "copy V");
    LR_CUDA(h, cudaStreamSynchronize(stm), "lr_truncate copy");
  }
  X->r = R;
  if (h->h_state->status) return fail(h, static_cast<lr_status>(h->h_state->status), kNonFiniteMsg);
  if (h->h_state->cut) return fail(h, LR_ENOCONV, "rank exceeds rmax; result truncated");
  return LR_OK;
}

}  // extern "C"
