// C ABI of liblrpoisson.so: handle, plan cache, workspace and the entry points
// declared in include/lrpoisson.h.  Every numerical step runs in the kernels of
// dst.cu, cross.cu and core.cu; this file validates arguments, lays out the
// workspace and enqueues the launches on the handle's stream.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "lr_internal.h"

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
  lr_info info{};
  int last_kcap = 0;
  cudaEvent_t ev[LR_NUM_PHASES + 1] = {};
  bool timed = false;
  // batched solves: internal streams, fork/join events, pinned status array
  cudaStream_t bstreams[16] = {};
  cudaEvent_t bjoin[16] = {};
  cudaEvent_t bfork = nullptr;
  SolveState* h_bstate = nullptr;
  int bstate_cap = 0;
  // captured CUDA graphs (LR_FLAG_GRAPH), keyed by every pointer and size
  cudaStream_t cap_stream = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  unsigned long long ws_gen = 0;
  int last_cs = 0;
};

namespace {

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

lr_status ensure_ws(lr_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return LR_OK;
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

// Enqueue T1-T6 of one solve on stream stm.  ev (optional) receives the
// phase boundaries.
template <typename T>
cudaError_t enqueue_solve(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options& o, const Plan& plan,
                          const SolveGeom& g, const Slice<T>& w, SolveState* st, cudaStream_t stm,
                          cudaEvent_t* ev, int* used_cs) {
  const bool f32 = sizeof(T) == 4;
  cudaError_t e;
  if ((e = cudaMemsetAsync(st, 0, sizeof(SolveState), stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[0], stm)) != cudaSuccess) return e;
  // T1: forward DST of both factors.
  ColumnSet fw;
  fw.in[0] = rhs->U; fw.in[1] = rhs->V;
  fw.ld_in[0] = rhs->ld; fw.ld_in[1] = rhs->ld;
  fw.out[0] = w.Uh; fw.out[1] = w.Vh;
  fw.ld_out[0] = g.ldw; fw.ld_out[1] = g.ldw;
  fw.ncol[0] = g.r; fw.ncol[1] = g.r;
  if ((e = launch_dst<T>(plan, fw, IoType::F64, IoType::WORK, w.work, h->num_sms, stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], stm)) != cudaSuccess) return e;
  // T2-T4: cross approximation in frequency space.
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
  // T5: rounding core.
  CoreArgs<T> co;
  co.GC = w.GC; co.GR = w.GR; co.ldg = g.kcap; co.d = w.d;
  co.k_dev = &st->k; co.k_host = 0;
  co.eps = o.eps; co.rmax_out = g.ncap_out;
  co.Tc = w.Tc; co.Tr = w.Tr; co.s_out = sol->s; co.st = st;
  if ((e = launch_core<T>(co, f32, stm)) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], stm)) != cudaSuccess) return e;
  // T6: inverse DST of the kept columns into the caller's float64 factors;
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
      for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
      h->graphs.clear();
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
  if (!hs.converged) return fail(h, LR_ENOCONV, "cross did not converge within opt->rmax steps");
  if (hs.cut) return fail(h, LR_ENOCONV, "solution rank exceeds sol->rmax; result truncated");
  return LR_OK;
}

constexpr int kBatchStreams = 16;

lr_status ensure_batch_streams(lr_handle h) {
  if (h->bstreams[0]) return LR_OK;
  for (int i = 0; i < kBatchStreams; ++i) {
    LR_CUDA(h, cudaStreamCreateWithFlags(&h->bstreams[i], cudaStreamNonBlocking), "stream create");
    LR_CUDA(h, cudaEventCreateWithFlags(&h->bjoin[i], cudaEventDisableTiming), "event create");
  }
  LR_CUDA(h, cudaEventCreateWithFlags(&h->bfork, cudaEventDisableTiming), "event create");
  return LR_OK;
}

template <typename T>
lr_status solve2d_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options& o,
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
      if ((e = enqueue_solve<T>(h, &rhs[i], &sol[i], o, *plans[i], geo[i], w, &states[i],
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
  lr_status worst = LR_OK;
  for (int i = 0; i < batch; ++i) {
    const SolveState& hs = h->h_bstate[i];
    sol[i].r = hs.rank;
    const lr_status si = (!hs.converged || hs.cut) ? LR_ENOCONV : LR_OK;
    if (per_problem) per_problem[i] = si;
    if (si != LR_OK) worst = si;
  }
  if (worst != LR_OK) fail(h, worst, "some problems did not converge or were cut (see per_problem)");
  return worst;
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
}

const char* lr_status_string(lr_status s) {
  switch (s) {
    case LR_OK: return "LR_OK";
    case LR_EINVAL: return "LR_EINVAL";
    case LR_ENOMEM: return "LR_ENOMEM";
    case LR_ENOCONV: return "LR_ENOCONV";
    case LR_ETIMEOUT: return "LR_ETIMEOUT";
    case LR_ECUDA: return "LR_ECUDA";
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
      cudaMallocHost(&h->h_piv, sizeof(int) * 2 * KMAX) != cudaSuccess) {
    cudaGetLastError();
    if (h->h_state) cudaFreeHost(h->h_state);
    delete h;
    return LR_ENOMEM;
  }
  std::memset(h->h_state, 0, sizeof(SolveState));
  std::memset(h->h_piv, 0, sizeof(int) * 2 * KMAX);
  *out = h;
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
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int i = 0; i < 16; ++i) {
    if (h->bstreams[i]) cudaStreamDestroy(h->bstreams[i]);
    if (h->bjoin[i]) cudaEventDestroy(h->bjoin[i]);
  }
  if (h->bfork) cudaEventDestroy(h->bfork);
  if (h->h_bstate) cudaFreeHost(h->h_bstate);
  h->plans.clear();
  if (h->ws) cudaFree(h->ws);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_piv) cudaFreeHost(h->h_piv);
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

lr_status lr_poisson2d(lr_handle h, const lr_mat* rhs, lr_mat* sol, const lr_options* opt) {
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
  s = o.prec == LR_MIXED ? solve2d<float>(h, rhs, sol, o, plan) : solve2d<double>(h, rhs, sol, o, plan);
  h->info.status = s;
  return s;
}

lr_status lr_poisson2d_batched(lr_handle h, int batch, const lr_mat* rhs, lr_mat* sol, const lr_options* opt,
                               lr_status* per_problem) {
  if (!h) return LR_EINVAL;
  lr_options o;
  if (opt) o = *opt; else lr_options_default(&o);
  lr_status s = check_opts(h, o);
  if (s != LR_OK) return s;
  if (batch < 0 || (batch > 0 && (!rhs || !sol))) return fail(h, LR_EINVAL, "bad batch arguments");
  if (batch == 0) return LR_OK;
  if (o.flags & LR_FLAG_TIMING) return fail(h, LR_EINVAL, "LR_FLAG_TIMING is for single solves");
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
  s = o.prec == LR_MIXED ? solve2d_batched<float>(h, batch, rhs, sol, o, plans, per_problem)
                         : solve2d_batched<double>(h, batch, rhs, sol, o, plans, per_problem);
  h->info.status = s;
  return s;
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
  if (h->h_state->cut) return fail(h, LR_ENOCONV, "rank exceeds rmax; result truncated");
  return LR_OK;
}

}  // extern "C"
