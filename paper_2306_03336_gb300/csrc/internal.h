// internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/j2d5pt.h"

namespace j2d {

// One grid of a plan: interior sizes, layout and weights {W, E, S, C, N}.
struct GridDesc {
  int nx = 0, ny = 0;
  long pitch = 0;  // elements per row
  long off = 0;    // element offset of logical column 0
  int shape = 5;   // 5: the five-point stencil, w = {W, E, S, C, N}; 9: the 3x3 box, w in row order
  double w[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  size_t bytes(size_t elem) const { return (size_t)(ny + 2) * (size_t)pitch * elem; }
};

// The plan layout of an nx*ny grid (include/j2d5pt.h): logical column 0 at
// element offset 16/sizeof-1, so interior column 1 starts a 16-byte vector;
// rows padded to whole 16-byte vectors.  Weights left zero.
inline GridDesc plan_layout(j2d_dtype dt, int nx, int ny) {
  GridDesc g;
  const long vec = dt == J2D_F64 ? 2 : 4;
  g.nx = nx;
  g.ny = ny;
  g.off = vec - 1;
  g.pitch = ((g.off + nx + 2) + vec - 1) / vec * vec;
  return g;
}

// Geometry of the temporally blocked kernels (chosen by the planner / tuner).
struct DtbConfig {
  int algo = J2D_ALGO_ONESTEP;  // resolved algorithm
  int depth = 1;                // steps per on-chip visit (BANDS / TILES)
  int tile_wx = 4;              // TILES: strips across a tile
  int ctas = 0;                 // persistent grid size
  int rows = 0;                 // rows per warp strip
  int sweep = 1;                // TILES, FP32 forward: time steps per shared-memory sweep (1 or 2)
};

// Device scratch for the temporally blocked kernels.
struct DtbScratch {
  void *base = nullptr;
  size_t bytes = 0;
};

// Record a message for j2d5pt_last_error() on this thread; returns `st`.
j2d_status record_error(j2d_status st, const char *fmt, ...);

// Count of kernels launched by the library (j2d5pt_kernel_launches).
extern std::atomic<long> g_launches;
inline void note_launch(long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t launch_onestep(j2d_dtype dt, bool adj, const void *in, void *out, const GridDesc &g, int ipath,
                           cudaStream_t s);
// the ring of `in` into out, or into `count` grids `ostride` elements apart
cudaError_t launch_ring_copy(j2d_dtype dt, const void *in, void *out, const GridDesc &g, cudaStream_t s,
                             long count = 1, long ostride = 0);
long wgrad_partial_count(j2d_dtype dt, const GridDesc &g);
cudaError_t launch_wgrad(j2d_dtype dt, const void *u, const void *lam, double *dw, double *partials,
                         const GridDesc &g, cudaStream_t s);
cudaError_t launch_adjoint_wgrad(j2d_dtype dt, const void *u, const void *lam1, void *lam0, double *dw,
                                 double *partials, long max_partials, const GridDesc &g, int ipath, cudaStream_t s);
// rows x width elements from src (row stride spitch; device-accessible, e.g.
// pinned host memory) to dst (row stride dpitch)
cudaError_t launch_gather_rows(j2d_dtype dt, const void *src, long spitch, void *dst, long dpitch, long rows, long width,
                               cudaStream_t s);
// STREAM schedule (stream.cu): temporal blocking in the register file.
constexpr int kStreamMaxF32 = 12;  // steps per pass, at most
constexpr int kStreamMaxF64 = 8;
struct StreamGeom {
  int depth = 1;  // steps per pass (M)
  int G = 0;      // halo columns on each side of a band
  int vw = 0;     // stored columns per band
  int bands = 0;  // column bands
  int H = 0;      // rows stored per run
  int runs = 0;   // runs per band
};
int stream_max_depth(j2d_dtype dt);
bool stream_depth_ok(j2d_dtype dt, int m, int shape = 5);  // a kernel of m steps per pass exists
bool stream_keep_ok(j2d_dtype dt, int m);   // ... and one that keeps every state
StreamGeom stream_geometry(j2d_dtype dt, const GridDesc &g, int depth, int sms);
// The same for a given number of warps resident at once (host arithmetic only).
StreamGeom stream_geometry_warps(j2d_dtype dt, int nx, int ny, int depth, long warps);
cudaError_t launch_stream_pass(j2d_dtype dt, const void *in, void *out, const GridDesc &g, const StreamGeom &q, int m,
                               int ipath, int *status, cudaStream_t s, void *keep = nullptr, long keep_stride = 0);

cudaError_t measure_fma(j2d_dtype dt, double *rate);
cudaError_t measure_exact(double *rate);
cudaError_t measure_exact_box(double *rate);
cudaError_t measure_smem(double *bytes_per_s);

}  // namespace j2d
