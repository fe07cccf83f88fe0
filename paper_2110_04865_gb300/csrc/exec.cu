// Device-side round loop as a CUDA graph.
//
// One instantiated graph per (device, stream, tile shape) is built on first
// use and reused for every later computation on that stream.  Its kernels
// read all sizes and buffers from a device-resident DevState slot, which each
// call fills with one small kernel before launching the graph, so calls on
// the same stream are ordered and never share a slot concurrently.
//
//   init (p_i = i, r = identity, mask = 0)
//   while (hooks in the last round) {                 Algorithm 2, loop test
//     min-edge sweep                                  multilinear step, projection
//     if (live slots < tau * slots) compact            (edge list shrinks)
//     hook; tie break                                 hooking, tie breaking
//     while (some changed root's parent moved) jump   Algorithm 3
//     shortcut every vertex; round end
//   }
//   labels; exact sums
// The host waits once, after copying the state back.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace msf {

namespace {

struct Executor {
  int device = 0;
  DevState *slot = nullptr;       // device
  DevState *host_copy = nullptr;  // pinned host
  cudaGraphExec_t exec = nullptr;
};

std::mutex g_exec_mu;

// MSF_TRACE=1 prints the graph construction steps to stderr.
bool tracing() {
  static int t = -1;
  if (t < 0) {
    const char *e = std::getenv("MSF_TRACE");
    t = (e && e[0] == '1') ? 1 : 0;
  }
  return t == 1;
}
#define TRACE(...)                        \
  do {                                    \
    if (tracing()) {                      \
      std::fprintf(stderr, "[msf] " __VA_ARGS__); \
      std::fputc('\n', stderr);          \
      std::fflush(stderr);                \
    }                                     \
  } while (0)
std::map<std::tuple<int, uintptr_t, int, int, int, int>, Executor *> g_execs;

// Handle for a conditional node that will be added to the graph being
// captured on `s`.
int make_handle(cudaStream_t s, unsigned default_value, cudaGraphConditionalHandle *h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  TRACE("make_handle: capture info");
  MSF_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  TRACE("make_handle: status %d graph %p", (int)cs, (void *)g);
  MSF_CK(cudaGraphConditionalHandleCreate(h, g, default_value, cudaGraphCondAssignDefault));
  TRACE("make_handle: handle %llu", (unsigned long long)*h);
  return MSF_OK;
}

// Adds a conditional node at the capture point of `s`, makes it the only
// dependency of what is captured next, and returns its body graph(s)
// (two for an if/else).
int add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraph_t *body, cudaGraph_t *else_body = nullptr) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  TRACE("add_conditional: capture info");
  MSF_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  TRACE("add_conditional: status %d graph %p deps %zu", (int)cs, (void *)g, nd);
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = else_body ? 2 : 1;
  cudaGraphNode_t node;
  MSF_CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  TRACE("add_conditional: node added, bodies %p", (void *)prm.conditional.phGraph_out);
  *body = prm.conditional.phGraph_out[0];
  if (else_body) *else_body = prm.conditional.phGraph_out[1];
  MSF_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  TRACE("add_conditional: dependencies updated");
  return MSF_OK;
}

#define MSF_RC(x)             \
  do {                        \
    int _rc = (x);            \
    if (_rc) return _rc;      \
  } while (0)

// Complete shortcutting over the changed roots (Algorithm 3), then one
// gather for every vertex.  Captured on `a`; the jump loop's body on `b`.
int capture_csp(DevState *st, cudaStream_t a, cudaStream_t b) {
  cudaGraphConditionalHandle hj;
  MSF_RC(make_handle(a, 0, &hj));
  launch_jump_init(st, hj, a);
  cudaGraph_t jbody;
  MSF_RC(add_conditional(a, hj, cudaGraphCondTypeWhile, &jbody));
  MSF_CK(cudaStreamBeginCaptureToGraph(b, jbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_jump(st, hj, b);
  MSF_CK(cudaStreamEndCapture(b, &jbody));
  launch_shortcut_all(st, a);
  return MSF_OK;
}

// Complete shortcutting by full passes over all vertices.
int capture_full(DevState *st, cudaStream_t a, cudaStream_t b) {
  cudaGraphConditionalHandle hj;
  MSF_RC(make_handle(a, 0, &hj));
  launch_jump_init(st, hj, a);
  cudaGraph_t jbody;
  MSF_RC(add_conditional(a, hj, cudaGraphCondTypeWhile, &jbody));
  MSF_CK(cudaStreamBeginCaptureToGraph(b, jbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_short_full(st, hj, b);
  MSF_CK(cudaStreamEndCapture(b, &jbody));
  return MSF_OK;
}

int capture_round_body(DevState *st, cudaGraph_t body, cudaGraphConditionalHandle hround, int spl, int bps,
                       int mode, cudaStream_t c1, cudaStream_t c2, cudaStream_t c3) {
  TRACE("round body: begin capture (shortcut mode %d)", mode);
  MSF_CK(cudaStreamBeginCaptureToGraph(c1, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  if (mode == MSF_SHORTCUT_ORIGINAL) launch_starcheck(st, c1);
  launch_prow(st, mode == MSF_SHORTCUT_ORIGINAL, c1);
  launch_min_edge(st, spl, bps, options().prefetch, c1, options().pairwise);
  TRACE("round body: min-edge captured");
  if (mode != MSF_SHORTCUT_ORIGINAL) {
    // compaction, when the live slots fell below tau
    cudaGraphConditionalHandle hc;
    MSF_RC(make_handle(c1, 0, &hc));
    launch_compact_decide(st, hc, c1);
    cudaGraph_t cbody;
    MSF_RC(add_conditional(c1, hc, cudaGraphCondTypeIf, &cbody));
    MSF_CK(cudaStreamBeginCaptureToGraph(c2, cbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_compact(st, spl, bps, c2);
    MSF_CK(cudaStreamEndCapture(c2, &cbody));
    TRACE("round body: compaction captured");
  }
  // hooking with tie breaking
  launch_hook(st, c1);
  // shortcutting
  switch (mode) {
    case MSF_SHORTCUT_ORIGINAL:
      launch_starcheck(st, c1);
      launch_short_step(st, c1);
      break;
    case MSF_SHORTCUT_FULL:
      MSF_RC(capture_full(st, c1, c2));
      break;
    case MSF_SHORTCUT_OPTIMIZED: {
      cudaGraphConditionalHandle hos;
      MSF_RC(make_handle(c1, 0, &hos));
      launch_os_decide(st, hos, c1);
      cudaGraph_t tbody, ebody;
      MSF_RC(add_conditional(c1, hos, cudaGraphCondTypeIf, &tbody, &ebody));
      MSF_CK(cudaStreamBeginCaptureToGraph(c2, tbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      MSF_RC(capture_csp(st, c2, c3));
      MSF_CK(cudaStreamEndCapture(c2, &tbody));
      MSF_CK(cudaStreamBeginCaptureToGraph(c2, ebody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      MSF_RC(capture_full(st, c2, c3));
      MSF_CK(cudaStreamEndCapture(c2, &ebody));
      break;
    }
    default:
      MSF_RC(capture_csp(st, c1, c2));
      break;
  }
  TRACE("round body: shortcut captured");
  launch_round_end(st, hround, c1);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaStreamEndCapture(c1, &body));
  TRACE("round body: done");
  return MSF_OK;
}

int build_graph(Executor *ex, int spl, int bps, int mode) {
  cudaStream_t c[4];
  for (int i = 0; i < 4; ++i) MSF_CK(cudaStreamCreateWithFlags(&c[i], cudaStreamNonBlocking));
  DevState *st = ex->slot;
  cudaGraph_t top;
  MSF_CK(cudaGraphCreate(&top, 0));
  MSF_CK(cudaStreamBeginCaptureToGraph(c[0], top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_init(st, c[0]);
  cudaGraphConditionalHandle hround;
  MSF_RC(make_handle(c[0], 1, &hround));
  cudaGraph_t body;
  MSF_RC(add_conditional(c[0], hround, cudaGraphCondTypeWhile, &body));
  MSF_RC(capture_round_body(st, body, hround, spl, bps, mode, c[1], c[2], c[3]));
  launch_labels(st, c[0]);
  launch_sums(st, c[0]);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaStreamEndCapture(c[0], &top));
  TRACE("top: captured, instantiating");
  MSF_CK(cudaGraphInstantiate(&ex->exec, top, 0));
  TRACE("top: instantiated");
  MSF_CK(cudaGraphDestroy(top));
  for (int i = 0; i < 4; ++i) cudaStreamDestroy(c[i]);
  return MSF_OK;
}

// Connected components (Sec. 2.4) with complete shortcutting by full passes:
//   init; while (some root hooked) { conditional sweep + hook; starcheck;
//   unconditional sweep (stars only) + hook; full shortcut passes; round end }
//   labels.
int build_cc_graph(Executor *ex) {
  cudaStream_t c[3];
  for (int i = 0; i < 3; ++i) MSF_CK(cudaStreamCreateWithFlags(&c[i], cudaStreamNonBlocking));
  DevState *st = ex->slot;
  cudaGraph_t top;
  MSF_CK(cudaGraphCreate(&top, 0));
  MSF_CK(cudaStreamBeginCaptureToGraph(c[0], top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_init(st, c[0]);
  cudaGraphConditionalHandle hround;
  MSF_RC(make_handle(c[0], 1, &hround));
  cudaGraph_t body;
  MSF_RC(add_conditional(c[0], hround, cudaGraphCondTypeWhile, &body));
  MSF_CK(cudaStreamBeginCaptureToGraph(c[1], body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_cc_sweep(st, true, c[1]);
  launch_cc_hook(st, c[1]);
  launch_starcheck(st, c[1]);
  launch_cc_sweep(st, false, c[1]);
  launch_cc_hook(st, c[1]);
  MSF_RC(capture_full(st, c[1], c[2]));
  launch_round_end(st, hround, c[1]);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaStreamEndCapture(c[1], &body));
  launch_labels(st, c[0]);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaStreamEndCapture(c[0], &top));
  MSF_CK(cudaGraphInstantiate(&ex->exec, top, 0));
  MSF_CK(cudaGraphDestroy(top));
  for (int i = 0; i < 3; ++i) cudaStreamDestroy(c[i]);
  return MSF_OK;
}

std::mutex g_cc_mu;
std::map<std::pair<int, uintptr_t>, Executor *> g_cc_execs;

}  // namespace

int enqueue_cc_graph(const DevState &hs, cudaStream_t s, const DevState **host_state) {
  int dev = 0;
  MSF_CK(cudaGetDevice(&dev));
  Executor *ex = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_cc_mu);
    auto key = std::make_pair(dev, (uintptr_t)s);
    auto it = g_cc_execs.find(key);
    if (it != g_cc_execs.end()) {
      ex = it->second;
    } else {
      ex = new Executor();
      ex->device = dev;
      MSF_CK(cudaMalloc(&ex->slot, sizeof(DevState)));
      MSF_CK(cudaMallocHost(&ex->host_copy, sizeof(DevState)));
      int rc = build_cc_graph(ex);
      if (rc) {
        cudaFree(ex->slot);
        cudaFreeHost(ex->host_copy);
        delete ex;
        return rc;
      }
      g_cc_execs[key] = ex;
    }
  }
  DevState hg = hs;
  hg.use_graph = 1;
  launch_load_state(ex->slot, hg, s);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaGraphLaunch(ex->exec, s));
  MSF_CK(cudaMemcpyAsync(ex->host_copy, ex->slot, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  *host_state = ex->host_copy;
  return MSF_OK;
}

// Enqueues the round loop for the state `hs` on stream `s`, followed by a
// copy of the final state into *host_state (pinned, owned by the executor;
// valid after the caller synchronizes `s`).
int enqueue_msf_graph(const DevState &hs, cudaStream_t s, const DevState **host_state) {
  int dev = 0;
  MSF_CK(cudaGetDevice(&dev));
  const Options &o = options();
  Executor *ex = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_exec_mu);
    auto key = std::make_tuple(dev, (uintptr_t)s, o.spl, o.blocks_per_sm * 2 + o.prefetch, o.shortcut_mode,
                               o.pairwise * 2 + o.sweep);
    auto it = g_execs.find(key);
    if (it != g_execs.end()) {
      ex = it->second;
    } else {
      ex = new Executor();
      ex->device = dev;
      MSF_CK(cudaMalloc(&ex->slot, sizeof(DevState)));
      MSF_CK(cudaMallocHost(&ex->host_copy, sizeof(DevState)));
      int rc = build_graph(ex, o.spl, o.blocks_per_sm, o.shortcut_mode);
      if (rc) {
        cudaFree(ex->slot);
        cudaFreeHost(ex->host_copy);
        delete ex;
        return rc;
      }
      g_execs[key] = ex;
    }
  }
  TRACE("enqueue: load state (%zu bytes)", sizeof(DevState));
  DevState hg = hs;
  hg.use_graph = 1;
  launch_load_state(ex->slot, hg, s);
  MSF_CK(cudaGetLastError());
  TRACE("enqueue: launch graph");
  MSF_CK(cudaGraphLaunch(ex->exec, s));
  MSF_CK(cudaMemcpyAsync(ex->host_copy, ex->slot, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  *host_state = ex->host_copy;
  return MSF_OK;
}

// The same round loop driven from the host, one launch per kernel, with a
// synchronisation at every decision (used to profile the kernels one by one;
// MSF_EXEC=host).  Synchronizes `s`.
int run_host_loop(const DevState &hs, cudaStream_t s, const DevState **host_state) {
  static std::mutex mu;
  static std::map<int, Executor *> slots;
  int dev = 0;
  MSF_CK(cudaGetDevice(&dev));
  Executor *ex = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = slots.find(dev);
    if (it == slots.end()) {
      ex = new Executor();
      MSF_CK(cudaMalloc(&ex->slot, sizeof(DevState)));
      MSF_CK(cudaMallocHost(&ex->host_copy, sizeof(DevState)));
      slots[dev] = ex;
    } else {
      ex = it->second;
    }
  }
  const Options &o = options();
  DevState *st = ex->slot;
  DevState hh = hs;
  hh.use_graph = 0;
  auto read_ctl = [&](int32_t *field) -> int {
    const size_t off = (const char *)field - (const char *)ex->host_copy;
    MSF_CK(cudaMemcpyAsync((char *)ex->host_copy + off, (const char *)st + off, sizeof(int32_t),
                           cudaMemcpyDeviceToHost, s));
    MSF_CK(cudaStreamSynchronize(s));
    return MSF_OK;
  };
  const int mode = o.shortcut_mode;
  launch_load_state(st, hh, s);
  launch_init(st, s);
  for (;;) {
    if (mode == MSF_SHORTCUT_ORIGINAL) launch_starcheck(st, s);
    launch_prow(st, mode == MSF_SHORTCUT_ORIGINAL, s);
    launch_min_edge(st, o.spl, o.blocks_per_sm, o.prefetch, s, o.pairwise);
    if (mode != MSF_SHORTCUT_ORIGINAL) {
      launch_compact_decide(st, 0, s);
      MSF_RC(read_ctl(&ex->host_copy->ctl_compact));
      if (ex->host_copy->ctl_compact) launch_compact(st, o.spl, o.blocks_per_sm, s);
    }
    launch_hook(st, s);
    bool csp = mode == MSF_SHORTCUT_CSP;
    if (mode == MSF_SHORTCUT_OPTIMIZED) {
      launch_os_decide(st, 0, s);
      MSF_RC(read_ctl(&ex->host_copy->ctl_compact));
      csp = ex->host_copy->ctl_compact != 0;
    }
    if (mode == MSF_SHORTCUT_ORIGINAL) {
      launch_starcheck(st, s);
      launch_short_step(st, s);
    } else {
      launch_jump_init(st, 0, s);
      MSF_RC(read_ctl(&ex->host_copy->ctl_jump));
      while (ex->host_copy->ctl_jump) {
        if (csp) launch_jump(st, 0, s);
        else launch_short_full(st, 0, s);
        MSF_RC(read_ctl(&ex->host_copy->ctl_jump));
      }
      if (csp) launch_shortcut_all(st, s);
    }
    launch_round_end(st, 0, s);
    MSF_RC(read_ctl(&ex->host_copy->ctl_round));
    if (!ex->host_copy->ctl_round) break;
  }
  launch_labels(st, s);
  launch_sums(st, s);
  MSF_CK(cudaGetLastError());
  MSF_CK(cudaMemcpyAsync(ex->host_copy, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  *host_state = ex->host_copy;
  return MSF_OK;
}

// The rest of one round from an externally reduced projection
// (msf_apply_round): hooking and tie breaking over every vertex, the chase of
// the changed roots (host-driven, a wait per pass), one gather for every
// vertex, the round's bookkeeping, the forest edges into the mask and, when
// asked for, the labels.  Uses a temporary state slot; synchronizes `s`.
int run_apply_round(const DevState &hs, cudaStream_t s, DevState *out) {
  int err = MSF_OK;
  DevState *slot = (DevState *)pool_alloc(sizeof(DevState), &err);
  if (err) return err;
  auto fin = [&](cudaError_t e) -> int {
    pool_free(slot);
    return e == cudaSuccess ? MSF_OK : cuda_fail(e, "apply round");
  };
  DevState hh = hs;
  hh.use_graph = 0;
  launch_load_state(slot, hh, s);
  launch_hook(slot, s);
  launch_jump_init(slot, 0, s);
  int32_t more = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&more, &slot->ctl_jump, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  while (e == cudaSuccess && more) {
    // k_jump_end bounds the passes by the jump limit
    launch_jump(slot, 0, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&more, &slot->ctl_jump, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return fin(e);
  launch_shortcut_all(slot, s);
  launch_round_end(slot, 0, s);
  launch_mask_from_keys(slot, s);
  if (hh.labels) launch_labels(slot, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, slot, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return fin(e);
}

// One min-edge sweep of the original CSR with a caller-supplied parent
// vector (msf_min_edge).  Uses a temporary state slot; synchronizes `s`.
// *ms receives the sweep's duration (CUDA events around that launch only).
int run_min_edge_once(const DevState &hs, cudaStream_t s, float *ms) {
  int err = MSF_OK;
  DevState *slot = (DevState *)pool_alloc(sizeof(DevState), &err);
  if (err) return err;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch_load_state(slot, hs, s);
    launch_prow(slot, 0, s);
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    // the timed unit is the sweep (the per-row parents were written before)
    launch_min_edge(slot, options().spl, options().blocks_per_sm, options().prefetch, s, options().pairwise);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  DevState back;
  if (e == cudaSuccess) e = cudaMemcpy(&back, slot, sizeof(DevState), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  pool_free(slot);
  if (e != cudaSuccess) return cuda_fail(e, "min-edge sweep");
  if (back.status) return fail(back.status, "min-edge sweep reported an inconsistent CSR");
  return MSF_OK;
}

}  // namespace msf
