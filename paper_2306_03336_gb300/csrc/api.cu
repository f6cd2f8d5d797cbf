// api.cu -- the C ABI (include/j2d5pt.h): plans, validation, workspace,
// dispatch to the one-step and temporally blocked kernels, host end-to-end
// runs, status reporting.
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "dtb.h"
#include "internal.h"

using namespace j2d;

static thread_local std::string g_last_error;

static j2d_status fail(j2d_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}
namespace j2d {
j2d_status record_error(j2d_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}
}  // namespace j2d

static j2d_status cuda_fail(cudaError_t e, const char *what) {
  return fail(J2D_ERR_DEVICE, "%s: %s", what, cudaGetErrorString(e));
}

struct j2d5pt_plan_s {
  int device = 0;
  j2d_dtype dtype = J2D_F64;
  size_t elem = 8;
  std::vector<GridDesc> grids;
  // options
  int opt_algo = J2D_ALGO_AUTO, opt_depth = 0, opt_tile_wx = 0, opt_ctas = 0, opt_verbose = 0;
  int opt_timeout_ms = 2000;
  int opt_fault = 0;
  int opt_int_path = 1;  // FP64 cells of the kExactMask pattern on the integer pipes
  int opt_sweep_steps = 2;  // FP32 tiles, forward: time steps per shared-memory sweep
  // device info
  int sms = 0;
  size_t smem_optin = 0;
  // workspace: one extra buffer per grid (ping-pong), weight-gradient partials, status word
  void *ws = nullptr;
  std::vector<size_t> ws_off;
  double *partials = nullptr;
  long max_partials = 0;  // capacity of `partials` in 5-double blocks
  int *d_status = nullptr;
  // host end-to-end staging (device buffers), allocated on first use
  void *h_in_dev = nullptr, *h_out_dev = nullptr;
  // scratch of the temporally blocked kernels
  DtbState dtb;
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  // kernel timing events (J2D_OPT_TIMING)
  int opt_timing = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  // CUDA graph of the last forward run (J2D_OPT_GRAPH)
  int opt_graph = 0;
  std::vector<const void *> g_in;
  std::vector<void *> g_out;
  long g_steps = -1;
  cudaGraphExec_t g_exec = nullptr;
  cudaStream_t g_stream = nullptr;
};

// Whether a plan's runs put the kExactMask cells on the integer path (FP64 only).
static int int_path_of(const j2d5pt_plan_s *p) { return p->dtype == J2D_F64 && p->opt_int_path ? 1 : 0; }

static void drop_graph(j2d5pt_plan_t p) {
  if (p->g_exec) cudaGraphExecDestroy(p->g_exec);
  p->g_exec = nullptr;
  p->g_in.clear();
  p->g_out.clear();
  p->g_steps = -1;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static j2d_status plan_common(j2d5pt_plan_t *out, int count, const int *nx, const int *ny, j2d_dtype dt,
                              const double *w, int shape = 5) {
  if (!out) return fail(J2D_ERR_ARG, "plan: null output pointer");
  *out = nullptr;
  if (dt != J2D_F64 && dt != J2D_F32) return fail(J2D_ERR_ARG, "plan: unknown dtype %d", (int)dt);
  if (count < 1 || !nx || !ny || !w) return fail(J2D_ERR_ARG, "plan: need count >= 1 and non-null sizes/weights");
  for (int i = 0; i < count; ++i) {
    if (nx[i] < 1 || ny[i] < 1) return fail(J2D_ERR_ARG, "plan: grid %d has nx=%d ny=%d (need >= 1)", i, nx[i], ny[i]);
    if ((long)nx[i] + 8 > (1L << 30) || (long)ny[i] + 8 > (1L << 30))
      return fail(J2D_ERR_ARG, "plan: grid %d too large", i);
    for (int d = 0; d < shape; ++d)
      if (!std::isfinite(w[shape * i + d])) return fail(J2D_ERR_ARG, "plan: grid %d weight %d is not finite", i, d);
  }
  auto *p = new j2d5pt_plan_s();
  p->dtype = dt;
  p->elem = dt == J2D_F64 ? 8 : 4;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "plan: cudaGetDevice"); }
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, p->device)) != cudaSuccess) { delete p; return cuda_fail(e, "plan: properties"); }
  p->sms = prop.multiProcessorCount;
  // the checked build keeps static shared memory per block (its bound-test
  // range, padded to the 1024-byte alignment of the dynamic shared memory)
  p->smem_optin = prop.sharedMemPerBlockOptin - (kChecked ? 1024 : 0);
  size_t ws_bytes = 0;
  long max_partials = 0;
  for (int i = 0; i < count; ++i) {
    GridDesc g = plan_layout(dt, nx[i], ny[i]);
    g.shape = shape;
    for (int d = 0; d < shape; ++d) g.w[d] = dt == J2D_F64 ? w[shape * i + d] : (double)(float)w[shape * i + d];
    p->grids.push_back(g);
    p->ws_off.push_back(ws_bytes);
    ws_bytes += (g.bytes(p->elem) + 255) / 256 * 256;
    long np = wgrad_partial_count(dt, g);
    if (np > max_partials) max_partials = np;
  }
  // room for a persistent grid of the fused adjoint step (up to 8 blocks per SM)
  max_partials = std::max<long>(max_partials, 8L * std::max(p->sms, 1));
  p->max_partials = max_partials;
  if ((e = cudaMalloc(&p->ws, ws_bytes)) != cudaSuccess) { delete p; return fail(J2D_ERR_NOMEM, "plan: workspace of %zu bytes: %s", ws_bytes, cudaGetErrorString(e)); }
  if ((e = cudaMalloc(&p->partials, sizeof(double) * 5 * (size_t)max_partials + 64)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_status, 64)) != cudaSuccess || (e = cudaMemset(p->d_status, 0, 64)) != cudaSuccess) {
    cudaFree(p->ws);
    cudaFree(p->partials);
    cudaFree(p->d_status);
    delete p;
    return fail(J2D_ERR_NOMEM, "plan: small buffers: %s", cudaGetErrorString(e));
  }
  *out = p;
  g_last_error.clear();
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_plan(j2d5pt_plan_t *plan, int nx, int ny, j2d_dtype dtype, const double weights[5]) {
  return plan_common(plan, 1, &nx, &ny, dtype, weights);
}

extern "C" j2d_status j2d5pt_plan_batched(j2d5pt_plan_t *plan, int count, const int *nx, const int *ny,
                                          j2d_dtype dtype, const double *weights) {
  return plan_common(plan, count, nx, ny, dtype, weights);
}

extern "C" j2d_status j2d9pt_plan(j2d5pt_plan_t *plan, int nx, int ny, j2d_dtype dtype, const double weights[9]) {
  return plan_common(plan, 1, &nx, &ny, dtype, weights, 9);
}

// The 3x3 box stencil is forward only: its plans refuse the adjoint, the
// weight gradient and the five-weight setter.
static bool is_box(j2d5pt_plan_t p) { return p->grids[0].shape == 9; }

extern "C" j2d_status j2d5pt_plan_destroy(j2d5pt_plan_t p) {
  if (!p) return fail(J2D_ERR_ARG, "destroy: null plan");
  if (p->ran && p->last_stream) cudaStreamSynchronize(p->last_stream);
  drop_graph(p);
  if (p->g_stream) cudaStreamDestroy(p->g_stream);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  dtb_release(p->dtb);
  cudaFree(p->ws);
  cudaFree(p->partials);
  cudaFree(p->d_status);
  cudaFree(p->h_in_dev);
  cudaFree(p->h_out_dev);
  delete p;
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_set_weights(j2d5pt_plan_t p, int index, const double *w) {
  if (!p || !w) return fail(J2D_ERR_ARG, "set_weights: null argument");
  if (is_box(p)) return fail(J2D_ERR_UNSUPPORTED, "set_weights: a 3x3 box plan has nine weights; make a new plan");
  if (index < 0 || index >= (int)p->grids.size()) return fail(J2D_ERR_ARG, "set_weights: index %d out of range", index);
  for (int d = 0; d < 5; ++d)
    if (!std::isfinite(w[d])) return fail(J2D_ERR_ARG, "set_weights: weight %d is not finite", d);
  for (int d = 0; d < 5; ++d) p->grids[index].w[d] = p->dtype == J2D_F64 ? w[d] : (double)(float)w[d];
  drop_graph(p);
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_layout(j2d5pt_plan_t p, int index, long *pitch, long *offset) {
  if (!p) return fail(J2D_ERR_ARG, "layout: null plan");
  if (index < 0 || index >= (int)p->grids.size()) return fail(J2D_ERR_ARG, "layout: index %d out of range", index);
  if (pitch) *pitch = p->grids[index].pitch;
  if (offset) *offset = p->grids[index].off;
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_set_option(j2d5pt_plan_t p, j2d_option opt, long v) {
  if (!p) return fail(J2D_ERR_ARG, "set_option: null plan");
  switch (opt) {
    case J2D_OPT_ALGO:
      if (v < J2D_ALGO_AUTO || v > J2D_ALGO_STREAM) return fail(J2D_ERR_ARG, "set_option: bad algo %ld", v);
      p->opt_algo = (int)v;
      drop_graph(p);
      break;
    case J2D_OPT_DEPTH:
      if (v < 0 || v > 256) return fail(J2D_ERR_ARG, "set_option: depth %ld outside 0..256", v);
      p->opt_depth = (int)v;
      drop_graph(p);
      break;
    case J2D_OPT_TILE_WX:
      if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8 && v != 16)
        return fail(J2D_ERR_ARG, "set_option: tile_wx must be 0, 1, 2, 4, 8 or 16");
      p->opt_tile_wx = (int)v;
      drop_graph(p);
      break;
    case J2D_OPT_CTAS:
      if (v < 0 || v > 65535) return fail(J2D_ERR_ARG, "set_option: ctas %ld", v);
      p->opt_ctas = (int)v;
      break;
    case J2D_OPT_TIMEOUT_MS:
      if (v < 1 || v > 600000) return fail(J2D_ERR_ARG, "set_option: timeout %ld ms", v);
      p->opt_timeout_ms = (int)v;
      break;
    case J2D_OPT_VERBOSE:
      p->opt_verbose = (int)v;
      break;
    case J2D_OPT_GRAPH:
      p->opt_graph = v != 0;
      drop_graph(p);
      break;
    case J2D_OPT_FAULT_INJECT:
      p->opt_fault = v != 0;
      drop_graph(p);
      break;
    case J2D_OPT_INT_PATH:
      if (v != 0 && v != 1) return fail(J2D_ERR_ARG, "set_option: int_path must be 0 or 1");
      p->opt_int_path = (int)v;
      drop_graph(p);
      break;
    case J2D_OPT_SWEEP_STEPS:
      if (v != 1 && v != 2) return fail(J2D_ERR_ARG, "set_option: sweep_steps must be 1 or 2");
      p->opt_sweep_steps = (int)v;
      drop_graph(p);
      break;
    case J2D_OPT_TIMING:
      p->opt_timing = v != 0;
      if (p->opt_timing && !p->ev0) {
        cudaEventCreate(&p->ev0);
        cudaEventCreate(&p->ev1);
      }
      drop_graph(p);
      break;
    default:
      return fail(J2D_ERR_ARG, "set_option: unknown option %d", (int)opt);
  }
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_get_option(j2d5pt_plan_t p, j2d_option opt, long *v) {
  if (!p || !v) return fail(J2D_ERR_ARG, "get_option: null argument");
  switch (opt) {
    case J2D_OPT_ALGO: *v = p->opt_algo; break;
    case J2D_OPT_DEPTH: *v = p->opt_depth; break;
    case J2D_OPT_TILE_WX: *v = p->opt_tile_wx; break;
    case J2D_OPT_CTAS: *v = p->opt_ctas; break;
    case J2D_OPT_TIMEOUT_MS: *v = p->opt_timeout_ms; break;
    case J2D_OPT_VERBOSE: *v = p->opt_verbose; break;
    case J2D_OPT_GRAPH: *v = p->opt_graph; break;
    case J2D_OPT_TIMING: *v = p->opt_timing; break;
    case J2D_OPT_FAULT_INJECT: *v = p->opt_fault; break;
    case J2D_OPT_INT_PATH: *v = p->opt_int_path; break;
    case J2D_OPT_SWEEP_STEPS: *v = p->opt_sweep_steps; break;
    default: return fail(J2D_ERR_ARG, "get_option: unknown option %d", (int)opt);
  }
  return J2D_OK;
}

// Resolve the configuration a run will use.
static DtbConfig resolve(j2d5pt_plan_t p, long steps, bool adj) {
  DtbRequest rq;
  rq.algo = p->opt_algo;
  rq.depth = p->opt_depth;
  rq.tile_wx = p->opt_tile_wx;
  rq.ctas = p->opt_ctas;
  rq.steps = steps;
  rq.adjoint = adj;
  rq.sweep_steps = p->opt_sweep_steps;
  return dtb_choose(p->dtype, p->grids, p->sms, p->smem_optin, rq);
}

static const char *algo_name(int a) {
  switch (a) {
    case J2D_ALGO_ONESTEP: return "onestep";
    case J2D_ALGO_RESIDENT: return "resident";
    case J2D_ALGO_BANDS: return "bands";
    case J2D_ALGO_TILES: return "tiles";
    case J2D_ALGO_SKEWED: return "skewed";
    case J2D_ALGO_STREAM: return "stream";
    default: return "auto";
  }
}

extern "C" j2d_status j2d5pt_describe(j2d5pt_plan_t p, char *buf, size_t len) {
  if (!p || !buf || len == 0) return fail(J2D_ERR_ARG, "describe: null argument");
  DtbConfig c = resolve(p, 1000, false);
  snprintf(buf, len, "dtype=%s grids=%zu nx=%d ny=%d pitch=%ld offset=%ld algo=%s depth=%d tile_wx=%d ctas=%d rows=%d sweep=%d sms=%d stencil=%s",
           p->dtype == J2D_F64 ? "f64" : "f32", p->grids.size(), p->grids[0].nx, p->grids[0].ny, p->grids[0].pitch,
           p->grids[0].off, algo_name(c.algo), c.depth, c.tile_wx, c.ctas, c.rows, c.sweep, p->sms,
           is_box(p) ? "box9" : "j2d5pt");
  return J2D_OK;
}

static char *ws_of(j2d5pt_plan_t p, int i) { return (char *)p->ws + p->ws_off[i]; }

// One grid, `steps` forward (or adjoint) steps, in -> out.
static j2d_status run_grid_onestep(j2d5pt_plan_t p, int gi, const void *in, void *out, long steps, bool adj,
                                   cudaStream_t s) {
  const GridDesc &g = p->grids[gi];
  const size_t bytes = g.bytes(p->elem);
  cudaError_t e;
  if (steps == 0) {
    if (in != out && (e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "run: copy");
    return J2D_OK;
  }
  void *ws = ws_of(p, gi);
  const void *src = in;
  if (in == out && (steps & 1)) {
    if ((e = cudaMemcpyAsync(ws, in, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return cuda_fail(e, "run: copy");
    src = ws;
  }
  // no timing events inside a stream capture (a captured event cannot be
  // synchronised on later)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  const bool timing = p->opt_timing && p->ev0 && gi == 0 && !capturing;
  if (timing) cudaEventRecord(p->ev0, s);
  for (long t = 0; t < steps; ++t) {
    void *dst = ((steps - 1 - t) % 2 == 0) ? out : ws;
    if ((e = launch_onestep(p->dtype, adj, src, dst, g, int_path_of(p), s)) != cudaSuccess)
      return cuda_fail(e, "run: one-step launch");
    src = dst;
  }
  if (p->opt_timing && p->ev1 && !capturing && gi == (int)p->grids.size() - 1) {
    cudaEventRecord(p->ev1, s);
    p->timed = true;
  }
  return J2D_OK;
}

static j2d_status run_dtb(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps, bool adj,
                          const DtbConfig &c, cudaStream_t s, void *states = nullptr, long state_elems = 0);

// One grid, `steps` forward steps, in -> out, by the STREAM schedule: ceil(steps
// / depth) passes between out and the plan's ping-pong buffer, the first pass
// taking the remainder; every buffer a pass writes first receives the input's ring.
static j2d_status run_grid_stream(j2d5pt_plan_t p, int gi, const void *in, void *out, long steps, int depth,
                                  cudaStream_t s) {
  const GridDesc &g = p->grids[gi];
  if (!stream_depth_ok(p->dtype, depth, g.shape))
    return fail(J2D_ERR_ARG, "run: no stream kernel of depth %d for %s%s", depth, p->dtype == J2D_F64 ? "f64" : "f32",
                g.shape == 9 ? " box" : "");
  const StreamGeom q = stream_geometry(p->dtype, g, depth, p->sms);
  const long passes = (steps + q.depth - 1) / q.depth;
  const int first = (int)(steps - (passes - 1) * q.depth);
  void *ws = ws_of(p, gi);
  const void *src = in;
  cudaError_t e;
  if (in == out && (passes & 1)) {
    if ((e = cudaMemcpyAsync(ws, in, g.bytes(p->elem), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "run: copy");
    src = ws;
  }
  if (out != in && (e = launch_ring_copy(p->dtype, in, out, g, s)) != cudaSuccess) return cuda_fail(e, "run: ring");
  if (passes >= 2 && src != ws && (e = launch_ring_copy(p->dtype, in, ws, g, s)) != cudaSuccess)
    return cuda_fail(e, "run: ring");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool timing = p->opt_timing && p->ev0 && cap == cudaStreamCaptureStatusNone;
  if (timing) cudaEventRecord(p->ev0, s);
  for (long j = 0; j < passes; ++j) {
    void *dst = ((passes - 1 - j) % 2 == 0) ? out : ws;
    if ((e = launch_stream_pass(p->dtype, src, dst, g, q, j == 0 ? first : q.depth, int_path_of(p), p->d_status,
                                s)) != cudaSuccess)
      return cuda_fail(e, "run: stream launch");
    src = dst;
  }
  if (timing) {
    cudaEventRecord(p->ev1, s);
    p->timed = true;
  }
  return J2D_OK;
}

static j2d_status run_common(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps, bool adj,
                             cudaStream_t s) {
  if (steps < 0) return fail(J2D_ERR_ARG, "run: steps %ld < 0", steps);
  for (size_t i = 0; i < p->grids.size(); ++i) {
    if (!in[i] || !out[i]) return fail(J2D_ERR_ARG, "run: null buffer for grid %zu", i);
    if (!aligned16(in[i]) || !aligned16(out[i])) return fail(J2D_ERR_ALIGN, "run: buffer for grid %zu not 16-byte aligned", i);
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) return fail(J2D_ERR_DEVICE, "run: current device %d differs from the plan's device %d", cur, p->device);
  DtbConfig c = resolve(p, steps, adj);
  if (p->opt_verbose)
    fprintf(stderr, "[j2d5pt] run steps=%ld adj=%d algo=%s depth=%d tile_wx=%d ctas=%d rows=%d\n", steps, (int)adj,
            algo_name(c.algo), c.depth, c.tile_wx, c.ctas, c.rows);
  p->last_stream = s;
  p->ran = true;
  if (c.algo == J2D_ALGO_ONESTEP || steps == 0) {
    for (size_t i = 0; i < p->grids.size(); ++i) {
      j2d_status st = run_grid_onestep(p, (int)i, in[i], out[i], steps, adj, s);
      if (st != J2D_OK) return st;
    }
    return J2D_OK;
  }
  if (c.algo == J2D_ALGO_STREAM) return run_grid_stream(p, 0, in[0], out[0], steps, c.depth, s);
  return run_dtb(p, in, out, steps, adj, c, s);
}

// One temporally blocked launch (with its set-up) for a resolved configuration;
// `states` (one grid, forward) keeps every state, `state_elems` apart.
static j2d_status run_dtb(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps, bool adj,
                          const DtbConfig &c, cudaStream_t s, void *states, long state_elems) {
  std::vector<void *> wsv;
  for (size_t i = 0; i < p->grids.size(); ++i) wsv.push_back(ws_of(p, (int)i));
  DtbRun r;
  r.dtype = p->dtype;
  r.grids = &p->grids;
  r.in = in;
  r.out = out;
  r.ws = wsv.data();
  r.steps = steps;
  r.adjoint = adj;
  r.cfg = c;
  r.states = states;
  r.state_elems = state_elems;
  r.status = p->d_status;
  r.timeout_ns = (unsigned long long)p->opt_timeout_ms * 1000000ull;
  r.mute_slot = p->opt_fault ? 0 : -1;
  r.int_path = int_path_of(p);
  r.sms = p->sms;
  r.smem_optin = p->smem_optin;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (p->opt_timing && p->ev0 && cap == cudaStreamCaptureStatusNone) {
    r.ev0 = p->ev0;
    r.ev1 = p->ev1;
    p->timed = true;
  }
  std::string err;
  cudaError_t e = dtb_run(p->dtb, r, s, err);
  if (e == cudaErrorNotSupported) return fail(J2D_ERR_UNSUPPORTED, "run: %s", err.c_str());
  if (e == cudaErrorMemoryAllocation) return fail(J2D_ERR_NOMEM, "run: %s", err.c_str());
  if (e != cudaSuccess) return fail(J2D_ERR_DEVICE, "run: %s: %s", err.c_str(), cudaGetErrorString(e));
  return J2D_OK;
}

// Forward run, through a CUDA graph when J2D_OPT_GRAPH is set: the first call
// for given buffers and step count runs normally (sizing the workspace and
// uploading the launch descriptors), then captures the same sequence of
// launches on a private stream; later identical calls replay the graph.
static j2d_status run_forward(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps, cudaStream_t s) {
  if (!p->opt_graph) return run_common(p, in, out, steps, false, s);
  const size_t n = p->grids.size();
  bool hit = p->g_exec && p->g_steps == steps;
  for (size_t i = 0; hit && i < n; ++i) hit = p->g_in[i] == in[i] && p->g_out[i] == out[i];
  cudaError_t e;
  if (hit) {
    if ((e = cudaGraphLaunch(p->g_exec, s)) != cudaSuccess) return cuda_fail(e, "run: graph launch");
    p->last_stream = s;
    p->ran = true;
    return J2D_OK;
  }
  drop_graph(p);
  j2d_status st = run_common(p, in, out, steps, false, s);
  if (st != J2D_OK || steps == 0) return st;
  if (!p->g_stream && (e = cudaStreamCreateWithFlags(&p->g_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "run: graph stream");
  // the capture stream must not start before the plain run has finished with the buffers
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "run: sync before capture");
  if ((e = cudaStreamBeginCapture(p->g_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(e, "run: begin capture");
  st = run_common(p, in, out, steps, false, p->g_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(p->g_stream, &graph);
  p->last_stream = s;
  if (st != J2D_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "run: end capture");
  e = cudaGraphInstantiate(&p->g_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    p->g_exec = nullptr;
    return cuda_fail(e, "run: graph instantiate");
  }
  p->g_in.assign(in, in + n);
  p->g_out.assign(out, out + n);
  p->g_steps = steps;
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_run(j2d5pt_plan_t p, const void *in, void *out, long steps, void *stream) {
  if (!p) return fail(J2D_ERR_ARG, "run: null plan");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "run: batched plan; use j2d5pt_run_batched");
  return run_forward(p, &in, &out, steps, (cudaStream_t)stream);
}

extern "C" j2d_status j2d5pt_run_batched(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps,
                                         void *stream) {
  if (!p || !in || !out) return fail(J2D_ERR_ARG, "run_batched: null argument");
  return run_forward(p, in, out, steps, (cudaStream_t)stream);
}

extern "C" j2d_status j2d5pt_run_adjoint(j2d5pt_plan_t p, const void *lam_T, void *lam_0, long steps, void *stream) {
  if (!p) return fail(J2D_ERR_ARG, "run_adjoint: null plan");
  if (is_box(p)) return fail(J2D_ERR_UNSUPPORTED, "run_adjoint: the 3x3 box stencil is forward only");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "run_adjoint: batched plans are forward only");
  return run_common(p, &lam_T, &lam_0, steps, true, (cudaStream_t)stream);
}

extern "C" j2d_status j2d5pt_weight_grad(j2d5pt_plan_t p, const void *u_t, const void *lam_t1, double *dw,
                                         void *stream) {
  if (!p || !u_t || !lam_t1 || !dw) return fail(J2D_ERR_ARG, "weight_grad: null argument");
  if (is_box(p)) return fail(J2D_ERR_UNSUPPORTED, "weight_grad: the 3x3 box stencil is forward only");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "weight_grad: batched plans are forward only");
  if (!aligned16(u_t) || !aligned16(lam_t1)) return fail(J2D_ERR_ALIGN, "weight_grad: buffer not 16-byte aligned");
  if (((uintptr_t)dw & 7u) != 0) return fail(J2D_ERR_ALIGN, "weight_grad: dw not 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  p->ran = true;
  cudaError_t e = launch_wgrad(p->dtype, u_t, lam_t1, dw, p->partials, p->grids[0], s);
  if (e != cudaSuccess) return cuda_fail(e, "weight_grad: launch");
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_adjoint_step_wgrad(j2d5pt_plan_t p, const void *u_t, const void *lam_t1, void *lam_t,
                                               double *dw, void *stream) {
  if (!p || !u_t || !lam_t1 || !lam_t || !dw) return fail(J2D_ERR_ARG, "adjoint_step_wgrad: null argument");
  if (is_box(p)) return fail(J2D_ERR_UNSUPPORTED, "adjoint_step_wgrad: the 3x3 box stencil is forward only");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "adjoint_step_wgrad: batched plans are forward only");
  if (lam_t == lam_t1 || lam_t == u_t) return fail(J2D_ERR_ARG, "adjoint_step_wgrad: lam_t aliases an input");
  if (!aligned16(u_t) || !aligned16(lam_t1) || !aligned16(lam_t))
    return fail(J2D_ERR_ALIGN, "adjoint_step_wgrad: buffer not 16-byte aligned");
  if (((uintptr_t)dw & 7u) != 0) return fail(J2D_ERR_ALIGN, "adjoint_step_wgrad: dw not 8-byte aligned");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) return fail(J2D_ERR_DEVICE, "adjoint_step_wgrad: current device %d differs from the plan's device %d", cur, p->device);
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  p->ran = true;
  cudaError_t e = launch_adjoint_wgrad(p->dtype, u_t, lam_t1, lam_t, dw, p->partials, p->max_partials, p->grids[0],
                                       int_path_of(p), s);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint_step_wgrad: launch");
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_run_host(j2d5pt_plan_t p, const void *h_in, void *h_out, long steps) {
  if (!p || !h_in || !h_out) return fail(J2D_ERR_ARG, "run_host: null argument");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "run_host: single-grid plans only");
  const GridDesc &g = p->grids[0];
  cudaError_t e;
  if (!p->h_in_dev) {
    if ((e = cudaMalloc(&p->h_in_dev, g.bytes(p->elem))) != cudaSuccess ||
        (e = cudaMalloc(&p->h_out_dev, g.bytes(p->elem))) != cudaSuccess) {
      cudaFree(p->h_in_dev);
      p->h_in_dev = nullptr;
      return fail(J2D_ERR_NOMEM, "run_host: staging buffers: %s", cudaGetErrorString(e));
    }
  }
  cudaStream_t s = nullptr;
  const size_t w = (size_t)(g.nx + 2) * p->elem, dp = (size_t)g.pitch * p->elem;
  char *din = (char *)p->h_in_dev + g.off * p->elem, *dout = (char *)p->h_out_dev + g.off * p->elem;
  // pinned (device-accessible) input: gathered by a kernel; otherwise one 2D copy
  cudaPointerAttributes pa{};
  const void *h_dev = nullptr;
  if (cudaPointerGetAttributes(&pa, h_in) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
    h_dev = pa.devicePointer;
  else
    cudaGetLastError();  // clear a failed query
  if (h_dev) {
    if ((e = launch_gather_rows(p->dtype, h_dev, g.nx + 2, din, g.pitch, g.ny + 2, g.nx + 2, s)) != cudaSuccess)
      return cuda_fail(e, "run_host: gather in");
  } else if ((e = cudaMemcpy2DAsync(din, dp, h_in, w, w, g.ny + 2, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    return cuda_fail(e, "run_host: copy in");
  }
  j2d_status st = j2d5pt_run(p, p->h_in_dev, p->h_out_dev, steps, s);
  if (st != J2D_OK) return st;
  if ((e = cudaMemcpy2DAsync(h_out, w, dout, dp, w, g.ny + 2, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "run_host: copy out");
  return j2d5pt_sync_status(p);
}

extern "C" j2d_status j2d5pt_run_states(j2d5pt_plan_t p, const void *in, void *states, long steps, void *stream) {
  if (!p || !in || !states) return fail(J2D_ERR_ARG, "run_states: null argument");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "run_states: single-grid plans only");
  if (is_box(p)) return fail(J2D_ERR_UNSUPPORTED, "run_states: five-point plans only");
  if (steps < 1) return fail(J2D_ERR_ARG, "run_states: steps must be >= 1");
  if (!aligned16(in) || !aligned16(states)) return fail(J2D_ERR_ALIGN, "run_states: buffer not 16-byte aligned");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) return fail(J2D_ERR_DEVICE, "run_states: current device %d differs from the plan's device %d", cur, p->device);
  const GridDesc &g = p->grids[0];
  const long se = (long)(g.ny + 2) * g.pitch;  // elements per state
  const size_t sb = (size_t)se * p->elem;
  char *st0 = (char *)states;
  if ((const char *)in >= st0 && (const char *)in < st0 + sb * (size_t)steps)
    return fail(J2D_ERR_ARG, "run_states: in lies inside states");
  cudaStream_t s = (cudaStream_t)stream;
  p->last_stream = s;
  p->ran = true;
  cudaError_t e;
  if ((e = launch_ring_copy(p->dtype, in, states, g, s, steps, se)) != cudaSuccess) return cuda_fail(e, "run_states: rings");
  // AUTO keeps the states with the one-step kernel, which writes every state
  // anyway: FP64 4096^2, 49 states, 6.48 ms against 6.81 for tiles storing
  // each step (the stores cost the tiled sweep 18%)
  DtbConfig c = resolve(p, steps, false);
  if (p->opt_algo == J2D_ALGO_AUTO) c.algo = J2D_ALGO_ONESTEP;
  if (c.algo == J2D_ALGO_ONESTEP) {
    const void *src = in;
    for (long t = 0; t < steps; ++t) {
      void *dst = st0 + (size_t)t * sb;
      if ((e = launch_onestep(p->dtype, false, src, dst, g, int_path_of(p), s)) != cudaSuccess)
        return cuda_fail(e, "run_states: one-step launch");
      src = dst;
    }
    return J2D_OK;
  }
  if (c.algo == J2D_ALGO_STREAM) {
    // the stream schedule stores every step's rows from its pipeline: passes
    // of k steps, pass j reading the state before it and writing its k states
    const int depth = stream_keep_ok(p->dtype, c.depth) ? c.depth : (p->dtype == J2D_F64 ? 2 : 8);
    const StreamGeom q = stream_geometry(p->dtype, g, depth, p->sms);
    const long passes = (steps + q.depth - 1) / q.depth;
    const void *src = in;
    long s0 = 0;  // states before this pass
    for (long j = 0; j < passes; ++j) {
      const int m = (int)(j == 0 ? steps - (passes - 1) * q.depth : q.depth);
      char *keep = st0 + (size_t)s0 * sb;
      if ((e = launch_stream_pass(p->dtype, src, keep + (size_t)(m - 1) * sb, g, q, m, int_path_of(p), p->d_status,
                                  s, keep, se)) != cudaSuccess)
        return cuda_fail(e, "run_states: stream launch");
      src = keep + (size_t)(m - 1) * sb;
      s0 += m;
    }
    return J2D_OK;
  }
  if (c.algo == J2D_ALGO_SKEWED || c.sweep == 2) {
    // the skewed and two-step sweeps hold no whole state of a strip between
    // their steps: single-step tiles (the plan's depth and shape if it chose
    // tiles)
    DtbRequest rq;
    rq.algo = J2D_ALGO_TILES;
    rq.depth = c.algo == J2D_ALGO_TILES ? p->opt_depth : 0;
    rq.tile_wx = c.algo == J2D_ALGO_TILES ? p->opt_tile_wx : 0;
    rq.ctas = p->opt_ctas;
    rq.steps = steps;
    rq.sweep_steps = 1;
    c = dtb_choose(p->dtype, p->grids, p->sms, p->smem_optin, rq);
  }
  void *last = st0 + (size_t)(steps - 1) * sb;
  return run_dtb(p, &in, &last, steps, false, c, s, states, se);
}

extern "C" j2d_status j2d5pt_sync_status(j2d5pt_plan_t p) {
  if (!p) return fail(J2D_ERR_ARG, "sync_status: null plan");
  cudaError_t e = p->ran ? cudaStreamSynchronize(p->last_stream) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "sync_status: stream");
  int st = 0;
  if ((e = cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "sync_status: read");
  if (st == 0) st = dtb_bounds_fault();
  if (st != 0) {
    cudaMemset(p->d_status, 0, sizeof(int));
    if (st == J2D_ERR_TIMEOUT) return fail(J2D_ERR_TIMEOUT, "device: a wait exceeded the time limit; results invalid");
    return fail((j2d_status)st, "device: bound check failed (code %d); results invalid", st);
  }
  return J2D_OK;
}

// Autotuner.  Candidates: the one-step kernel; the resident kernel when the
// grid fits on chip; bands, tiles and skewed tiles over temporal depths k
// (and tile shapes); the stream schedule over its steps per pass.
// Each is timed with CUDA events for min(steps, 64) steps, or more when that
// takes under 5 ms (best of two or three runs after a warm-up run); the
// fastest per step is kept in the plan.  With J2D_TUNE_CACHE set, results are
// read from / appended to that file, keyed by device, SM count, dtype, grid
// sizes and the step-count bucket.
static std::string tune_key(j2d5pt_plan_t p, long steps) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->device);
  std::string k = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) + "|" +
                  (p->dtype == J2D_F64 ? "f64" : "f32");
  unsigned long long h = 1469598103934665603ull;
  for (const GridDesc &g : p->grids) {
    h = (h ^ (unsigned long long)g.nx) * 1099511628211ull;
    h = (h ^ (unsigned long long)g.ny) * 1099511628211ull;
  }
  k += "|" + std::to_string(p->grids.size()) + "|" + std::to_string(h) + "|ip" + std::to_string(int_path_of(p)) +
       "|sw" + std::to_string(p->opt_sweep_steps) + "|s" + std::to_string(p->grids[0].shape);
  long b = 1;
  while (b < steps) b <<= 1;
  k += "|" + std::to_string(b);
  // the cache file separates fields by whitespace: the key holds none
  for (char &ch : k)
    if (ch == ' ' || ch == '\t') ch = '_';
  return k;
}

static bool tune_cache_lookup(const std::string &key, int *algo, int *depth, int *wx) {
  const char *path = getenv("J2D_TUNE_CACHE");
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[400];
    int a, d, w;
    if (sscanf(line, "%399s %d %d %d", k, &a, &d, &w) == 4 && key == k) {
      *algo = a; *depth = d; *wx = w;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void tune_cache_store(const std::string &key, int algo, int depth, int wx) {
  const char *path = getenv("J2D_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", key.c_str(), algo, depth, wx);
  fclose(f);
}

static j2d_status autotune_common(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps,
                                  cudaStream_t s) {
  std::string key = tune_key(p, steps);
  int ca, cd, cw;
  if (tune_cache_lookup(key, &ca, &cd, &cw)) {
    p->opt_algo = ca;
    p->opt_depth = cd;
    p->opt_tile_wx = cw;
    return J2D_OK;
  }
  struct Cand { int algo, depth, wx; };
  std::vector<Cand> cands;
  const long tsteps = std::min<long>(steps, 64);
  const bool single = p->grids.size() == 1;
  if (single) cands.push_back({J2D_ALGO_ONESTEP, 0, 0});
  {
    DtbRequest rq;
    rq.algo = J2D_ALGO_RESIDENT;
    rq.steps = steps;
    if (dtb_choose(p->dtype, p->grids, p->sms, p->smem_optin, rq).algo == J2D_ALGO_RESIDENT)
      cands.push_back({J2D_ALGO_RESIDENT, 0, 0});  // a batch: grouped resident (waves of grids on chip)
  }
  const int depths[] = {2, 4, 6, 8, 12, 16, 24, 32};
  const bool box = is_box(p);  // the box runs the one-step kernel or the skewed tiles
  for (int d : depths) {
    if (d > steps) break;
    if (single && !box) cands.push_back({J2D_ALGO_BANDS, d, 0});
    if (!box)
      for (int wx : {1, 2, 4}) cands.push_back({J2D_ALGO_TILES, d, wx});
    for (int wx : {2, 4, 8}) cands.push_back({J2D_ALGO_SKEWED, d, wx});
  }
  if (single)
    for (int d = 1; d <= stream_max_depth(p->dtype) && d <= steps; ++d)
      if (stream_depth_ok(p->dtype, d, p->grids[0].shape)) cands.push_back({J2D_ALGO_STREAM, d, 0});
  float best_ms = 1e30f;
  Cand best = {J2D_ALGO_AUTO, 0, 0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (const Cand &c : cands) {
    p->opt_algo = c.algo;
    p->opt_depth = c.depth;
    p->opt_tile_wx = c.wx;
    // warm-up run, timed: a candidate that takes under 5 ms for tsteps is
    // timed over proportionally more steps (up to `steps`), so that short
    // runs are not decided by noise; candidates compare by time per step
    cudaEventRecord(e0, s);
    if (run_common(p, in, out, tsteps, false, s) != J2D_OK) continue;
    cudaEventRecord(e1, s);
    float warm = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || j2d5pt_sync_status(p) != J2D_OK ||
        cudaEventElapsedTime(&warm, e0, e1) != cudaSuccess)
      continue;
    long n = tsteps;
    if (warm < 5.0f && tsteps < steps)
      n = std::min<long>(steps, (long)std::ceil(tsteps * 5.0 / std::max(warm, 0.05f)));
    const int nrep = warm < 20.0f ? 3 : 2;  // best of three short runs, two long ones
    float ms = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < nrep && ok; ++rep) {
      cudaEventRecord(e0, s);
      j2d_status st = run_common(p, in, out, n, false, s);
      cudaEventRecord(e1, s);
      ok = st == J2D_OK && cudaEventSynchronize(e1) == cudaSuccess && j2d5pt_sync_status(p) == J2D_OK;
      float m = 0;
      if (ok && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess && m < ms) ms = m;
    }
    if (!ok) continue;
    const float per_step = ms / (float)n;
    if (p->opt_verbose)
      fprintf(stderr, "[j2d5pt] tune algo=%d depth=%d wx=%d: %.3f ms for %ld steps\n", c.algo, c.depth, c.wx, ms, n);
    if (per_step < best_ms) {
      best_ms = per_step;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->opt_algo = best.algo;
  p->opt_depth = best.depth;
  p->opt_tile_wx = best.wx;
  tune_cache_store(key, best.algo, best.depth, best.wx);
  g_last_error.clear();
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_autotune(j2d5pt_plan_t p, const void *in, void *out, long steps, void *stream) {
  if (!p || !in || !out) return fail(J2D_ERR_ARG, "autotune: null argument");
  if (p->grids.size() != 1) return fail(J2D_ERR_ARG, "autotune: batched plan; use j2d5pt_autotune_batched");
  if (steps < 1) return fail(J2D_ERR_ARG, "autotune: steps must be >= 1");
  return autotune_common(p, &in, &out, steps, (cudaStream_t)stream);
}

extern "C" j2d_status j2d5pt_autotune_batched(j2d5pt_plan_t p, const void *const *in, void *const *out, long steps,
                                              void *stream) {
  if (!p || !in || !out) return fail(J2D_ERR_ARG, "autotune_batched: null argument");
  if (steps < 1) return fail(J2D_ERR_ARG, "autotune_batched: steps must be >= 1");
  return autotune_common(p, in, out, steps, (cudaStream_t)stream);
}

extern "C" j2d_status j2d5pt_kernel_time(j2d5pt_plan_t p, double *ms) {
  if (!p || !ms) return fail(J2D_ERR_ARG, "kernel_time: null argument");
  if (!p->opt_timing || !p->timed) return fail(J2D_ERR_ARG, "kernel_time: no timed run (set J2D_OPT_TIMING first)");
  cudaError_t e = cudaEventSynchronize(p->ev1);
  if (e != cudaSuccess) return cuda_fail(e, "kernel_time: sync");
  float f = 0;
  if ((e = cudaEventElapsedTime(&f, p->ev0, p->ev1)) != cudaSuccess) return cuda_fail(e, "kernel_time: elapsed");
  *ms = f;
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_measure_fma_rate(j2d_dtype dt, double *rate) {
  if (!rate || (dt != J2D_F64 && dt != J2D_F32)) return fail(J2D_ERR_ARG, "measure_fma_rate: bad argument");
  cudaError_t e = measure_fma(dt, rate);
  if (e != cudaSuccess) return cuda_fail(e, "measure_fma_rate");
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_measure_smem_bandwidth(double *bytes_per_s) {
  if (!bytes_per_s) return fail(J2D_ERR_ARG, "measure_smem_bandwidth: null pointer");
  cudaError_t e = measure_smem(bytes_per_s);
  if (e != cudaSuccess) return cuda_fail(e, "measure_smem_bandwidth");
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_measure_exact_rate(double *cells_per_s) {
  if (!cells_per_s) return fail(J2D_ERR_ARG, "measure_exact_rate: null pointer");
  cudaError_t e = measure_exact(cells_per_s);
  if (e != cudaSuccess) return cuda_fail(e, "measure_exact_rate");
  return J2D_OK;
}

extern "C" j2d_status j2d9pt_measure_exact_rate(double *cells_per_s) {
  if (!cells_per_s) return fail(J2D_ERR_ARG, "j2d9pt_measure_exact_rate: null pointer");
  cudaError_t e = measure_exact_box(cells_per_s);
  if (e != cudaSuccess) return cuda_fail(e, "j2d9pt_measure_exact_rate");
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_stream_geometry(int nx, int ny, j2d_dtype dtype, int shape, int depth, long resident_warps,
                                             long out[6]) {
  if (nx < 1 || ny < 1) return fail(J2D_ERR_ARG, "stream_geometry: nx=%d ny=%d (need >= 1)", nx, ny);
  if (dtype != J2D_F64 && dtype != J2D_F32) return fail(J2D_ERR_ARG, "stream_geometry: unknown dtype %d", (int)dtype);
  if (shape != 5 && shape != 9) return fail(J2D_ERR_ARG, "stream_geometry: shape %d (5 or 9)", shape);
  if (!out) return fail(J2D_ERR_ARG, "stream_geometry: null output");
  if (resident_warps < 1) return fail(J2D_ERR_ARG, "stream_geometry: resident_warps %ld < 1", resident_warps);
  if (!stream_depth_ok(dtype, depth, shape))
    return fail(J2D_ERR_ARG, "stream_geometry: no stream kernel of depth %d for this dtype and shape", depth);
  const StreamGeom q = stream_geometry_warps(dtype, nx, ny, depth, resident_warps);
  out[0] = q.depth;
  out[1] = q.G;
  out[2] = q.vw;
  out[3] = q.bands;
  out[4] = q.H;
  out[5] = q.runs;
  return J2D_OK;
}

extern "C" j2d_status j2d5pt_arith_info(unsigned *exact_mask, int *exact_guard) {
  if (exact_mask) *exact_mask = kExactMask;
  if (exact_guard) *exact_guard = kExactGuard;
  return J2D_OK;
}

extern "C" long j2d5pt_kernel_launches(void) { return g_launches.load(); }

extern "C" const char *j2d5pt_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *j2d5pt_version(void) {
  return kChecked ? "j2d5pt-gb300 0.2 (sm_103a, bounds-checked build)" : "j2d5pt-gb300 0.2 (sm_103a)";
}
