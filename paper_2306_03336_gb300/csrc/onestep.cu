// onestep.cu -- the one-step j2d5pt kernel (time loop on the host, every step
// streams the grid through HBM), plus the ring copy, the weight-gradient
// reduction and the FMA-rate probe.
//
// One-step kernel (Zhang et al., GPGPU'23, Section 3.1, Listing 1 with the
// pointers in global memory): each thread owns one 16-byte vector of columns
// and ROWS consecutive rows.  It loads its ROWS+2 rows into registers (the
// listing's column cache t[ILP+2]), takes the x-1 / x+1 neighbours across the
// vector boundary from the adjacent lane with a warp shuffle (lane 0 and lane
// 31 read the one value beyond the warp from L1), and writes ROWS results.
// Every cell of the logical array, ring included, is produced: ring and
// outside cells through the identity links (forward) or the transposed ring
// links (adjoint) of cell_links(), so one kernel serves both directions.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace j2d {

constexpr int kWarpsX = 8;  // warps side by side in a block

template <typename T, int V>
__device__ __forceinline__ void unpack(const typename VecOf<T>::type &v, T *o);
template <>
__device__ __forceinline__ void unpack<double, 2>(const double2 &v, double *o) { o[0] = v.x; o[1] = v.y; }
template <>
__device__ __forceinline__ void unpack<float, 4>(const float4 &v, float *o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ double2 pack(const double *o, double2 *) { return make_double2(o[0], o[1]); }
__device__ __forceinline__ float4 pack(const float *o, float4 *) { return make_float4(o[0], o[1], o[2], o[3]); }

// Sum the five per-thread accumulators of a (32 x kWarpsX) block in a fixed
// order (xor tree within a warp, then warps in order) into partials[block].
__device__ __forceinline__ void block_partials(const double (&acc)[5], double *partials) {
  __shared__ double red[kWarpsX][5];
  const int lane = threadIdx.x;
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    double s = acc[d];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[threadIdx.y][d] = s;
  }
  __syncthreads();
  if (threadIdx.y == 0 && lane < 5) {
    double s = 0.0;
    for (int wi = 0; wi < kWarpsX; ++wi) s += red[wi][lane];
    partials[(long)blockIdx.x * 5 + lane] = s;
  }
}

// WG (adjoint only): also accumulate the weight gradient of this step,
// sum over interior cells of in[i] * u[nbr_d(i)] (in = lam_t+1), into one
// partial sum per block, reduced in a fixed order.
template <typename T, bool ADJ, int ROWS, bool WG = false>
__global__ void __launch_bounds__(256) onestep_kernel(const T *__restrict__ in, T *__restrict__ out, long pitch,
                                                      int off, int nx, int ny, Weights<T> w, int ipath,
                                                      const T *__restrict__ uw = nullptr,
                                                      double *__restrict__ partials = nullptr) {
  constexpr int V = VecOf<T>::V;
  using VT = typename VecOf<T>::type;
  const int lane = threadIdx.x;
  const int H = ny + 2;
  // persistent: each warp takes work items (one warp-wide column strip x ROWS
  // rows) in a grid-stride loop; the grid is sized to the resident capacity
  const long ncs = (pitch + 32 * V - 1) / (32 * V);
  const long nitems = ncs * ((H + ROWS - 1) / ROWS);
  const long nwarps = (long)gridDim.x * kWarpsX;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long it = (long)blockIdx.x * kWarpsX + threadIdx.y; it < nitems; it += nwarps) {
  const long pc0 = ((it % ncs) * 32 + lane) * V;
  const bool live = pc0 < pitch;
  const int xl0 = (int)(pc0 - off);  // logical x of element 0
  const int y0 = (int)(it / ncs) * ROWS;

  T t[ROWS + 2][V];
#pragma unroll
  for (int r = 0; r < ROWS + 2; ++r) {
    const int y = y0 - 1 + r;
    if (live && y >= 0 && y < H) {
      unpack<T, V>(*reinterpret_cast<const VT *>(in + (long)y * pitch + pc0), t[r]);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) t[r][v] = T(0);
    }
  }
  T uu[WG ? ROWS + 2 : 1][V];
  if constexpr (WG) {
#pragma unroll
    for (int r = 0; r < ROWS + 2; ++r) {
      const int y = y0 - 1 + r;
      if (live && y >= 0 && y < H) {
        unpack<T, V>(*reinterpret_cast<const VT *>(uw + (long)y * pitch + pc0), uu[r]);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) uu[r][v] = T(0);
      }
    }
  }
  // Elements outside the logical array (row padding) read as zero.
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int x = xl0 + v;
    if (x < 0 || x > nx + 1) {
#pragma unroll
      for (int r = 0; r < ROWS + 2; ++r) {
        t[r][v] = T(0);
        if constexpr (WG) uu[r][v] = T(0);
      }
    }
  }

  Links<T> cw[V];  // links of this thread's columns on rows away from the ring
  ExactW cu[V];    // the same links unpacked for the integer path (FP64)
#pragma unroll
  for (int v = 0; v < V; ++v) {
    cw[v] = cell_links<T, ADJ>(xl0 + v, ADJ ? 2 : 1, nx, ny, w);
    if constexpr (std::is_same<T, double>::value) cu[v] = exact_weights(cw[v]);
  }

  const bool lval = live && (xl0 - 1 >= 0) && (xl0 - 1 <= nx + 1);
  const bool rval = live && (xl0 + V <= nx + 1);
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int y = y0 + r;
    if (y >= H) break;
    T left = __shfl_up_sync(0xffffffffu, t[r + 1][V - 1], 1);
    T right = __shfl_down_sync(0xffffffffu, t[r + 1][0], 1);
    if (lane == 0) left = lval ? in[(long)y * pitch + pc0 - 1] : T(0);
    if (lane == 31) right = rval ? in[(long)y * pitch + pc0 + V] : T(0);
    const bool mid = ADJ ? (y >= 2 && y <= ny - 1) : (y >= 1 && y <= ny);
    T o[V];
    if (mid) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T xm = v == 0 ? left : t[r + 1][v - 1];
        const T xp = v == V - 1 ? right : t[r + 1][v + 1];
        if constexpr (std::is_same<T, double>::value)
          o[v] = stencil_cell(cw[v], cu[v], exact_cell(xl0 + v, y, ipath != 0), xm, xp, t[r][v], t[r + 1][v], t[r + 2][v]);
        else
          o[v] = stencil(cw[v], xm, xp, t[r][v], t[r + 1][v], t[r + 2][v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T xm = v == 0 ? left : t[r + 1][v - 1];
        const T xp = v == V - 1 ? right : t[r + 1][v + 1];
        o[v] = stencil(cell_links<T, ADJ>(xl0 + v, y, nx, ny, w), xm, xp, t[r][v], t[r + 1][v], t[r + 2][v]);
      }
    }
    if (live) *reinterpret_cast<VT *>(out + (long)y * pitch + pc0) = pack(o, (VT *)nullptr);
    if constexpr (WG) {
      T ul = __shfl_up_sync(0xffffffffu, uu[r + 1][V - 1], 1);
      T ur = __shfl_down_sync(0xffffffffu, uu[r + 1][0], 1);
      if (lane == 0) ul = lval ? uw[(long)y * pitch + pc0 - 1] : T(0);
      if (lane == 31) ur = rval ? uw[(long)y * pitch + pc0 + V] : T(0);
      if (y >= 1 && y <= ny) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int x = xl0 + v;
          if (x < 1 || x > nx) continue;
          const double gv = (double)t[r + 1][v];
          acc[0] = fma(gv, (double)(v == 0 ? ul : uu[r + 1][v - 1]), acc[0]);
          acc[1] = fma(gv, (double)(v == V - 1 ? ur : uu[r + 1][v + 1]), acc[1]);
          acc[2] = fma(gv, (double)uu[r][v], acc[2]);
          acc[3] = fma(gv, (double)uu[r + 1][v], acc[3]);
          acc[4] = fma(gv, (double)uu[r + 2][v], acc[4]);
        }
      }
    }
  }
  }
  if constexpr (WG) block_partials(acc, partials);
}

// One step of the 3x3 box stencil (j2d9pt), the same layout as
// onestep_kernel: a warp takes a 32-vector column strip of ROWS rows,
// holding ROWS+2 rows in registers; every row's x-1 / x+1 neighbours come
// from the adjacent lane by shuffles (lanes 0 and 31 read the one value
// beyond the warp).  Ring and outside cells keep their value.
template <typename T, int ROWS>
__global__ void __launch_bounds__(256) onestep_box_kernel(const T *__restrict__ in, T *__restrict__ out, long pitch,
                                                          int off, int nx, int ny, Box9<T> b, int ipath) {
  constexpr int V = VecOf<T>::V;
  using VT = typename VecOf<T>::type;
  const int lane = threadIdx.x;
  const int H = ny + 2;
  const long ncs = (pitch + 32 * V - 1) / (32 * V);
  const long nitems = ncs * ((H + ROWS - 1) / ROWS);
  const long nwarps = (long)gridDim.x * kWarpsX;
  ExactWN<9> u{};
  if constexpr (std::is_same<T, double>::value) u = box_exact_weights(b);
  for (long it = (long)blockIdx.x * kWarpsX + threadIdx.y; it < nitems; it += nwarps) {
    const long pc0 = ((it % ncs) * 32 + lane) * V;
    const bool live = pc0 < pitch;
    const int xl0 = (int)(pc0 - off);  // logical x of element 0
    const int y0 = (int)(it / ncs) * ROWS;
    const bool lval = live && (xl0 - 1 >= 0) && (xl0 - 1 <= nx + 1);
    const bool rval = live && (xl0 + V <= nx + 1);
    // rows y0-1 .. y0+ROWS with their left / right neighbours
    T t[ROWS + 2][V], tl[ROWS + 2], tr[ROWS + 2];
#pragma unroll
    for (int r = 0; r < ROWS + 2; ++r) {
      const int y = y0 - 1 + r;
      const bool yin = y >= 0 && y < H;
      if (live && yin) {
        unpack<T, V>(*reinterpret_cast<const VT *>(in + (long)y * pitch + pc0), t[r]);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) t[r][v] = T(0);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int x = xl0 + v;
        if (x < 0 || x > nx + 1) t[r][v] = T(0);  // row padding reads as zero
      }
      tl[r] = __shfl_up_sync(0xffffffffu, t[r][V - 1], 1);
      tr[r] = __shfl_down_sync(0xffffffffu, t[r][0], 1);
      if (lane == 0) tl[r] = (lval && yin) ? in[(long)y * pitch + pc0 - 1] : T(0);
      if (lane == 31) tr[r] = (rval && yin) ? in[(long)y * pitch + pc0 + V] : T(0);
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int y = y0 + r;
      if (y >= H) break;
      T o[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int x = xl0 + v;
        if (y >= 1 && y <= ny && x >= 1 && x <= nx) {
          auto nb = [&](int rr, int d) -> T {
            const int e = v + d;
            return e < 0 ? tl[rr] : e >= V ? tr[rr] : t[rr][e];
          };
          o[v] = stencil_box_cell(b, u, exact_cell(x, y, ipath != 0), nb(r, -1), nb(r, 0), nb(r, 1), nb(r + 1, -1),
                                  nb(r + 1, 0), nb(r + 1, 1), nb(r + 2, -1), nb(r + 2, 0), nb(r + 2, 1));
        } else {
          o[v] = t[r + 1][v];  // ring and outside cells keep their value
        }
      }
      if (live) *reinterpret_cast<VT *>(out + (long)y * pitch + pc0) = pack(o, (VT *)nullptr);
    }
  }
}

// Copy the ring (rows 0 and ny+1, columns 0 and nx+1) of `in` to `out`.
template <typename T>
__global__ void ring_copy_kernel(const T *__restrict__ in, T *__restrict__ out, long pitch, int off, int nx,
                                 int ny, long ostride, long count) {
  // the ring of `in` into `count` outputs `ostride` elements apart (blockIdx.y over outputs)
  const int n_rows = 2 * (nx + 2), n = n_rows + 2 * ny;
  for (long c = blockIdx.y; c < count; c += gridDim.y) {
    T *o = out + c * ostride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      int y, x;
      if (i < n_rows) {
        y = (i < nx + 2) ? 0 : ny + 1;
        x = i % (nx + 2);
      } else {
        const int j = i - n_rows;
        y = 1 + (j >> 1);
        x = (j & 1) ? nx + 1 : 0;
      }
      const long e = (long)y * pitch + off + x;
      o[e] = in[e];
    }
  }
}

// Weight-gradient partial sums: per block, sum over its cells of
// lam[i] * u[nbr_d(i)] for d = x-1, x+1, y-1, centre, y+1, in FP64, reduced in
// a fixed order (thread order, xor tree, warp order) so results are
// reproducible.
template <typename T, int ROWS>
__global__ void __launch_bounds__(256) wgrad_kernel(const T *__restrict__ u, const T *__restrict__ lam, long pitch,
                                                    int off, int nx, int ny, double *__restrict__ partials) {
  constexpr int V = VecOf<T>::V;
  using VT = typename VecOf<T>::type;
  const int lane = threadIdx.x;
  // one work item per warp: a 32-vector column strip x ROWS interior rows,
  // numbered across the whole grid so no block covers only padding
  const long ncs = (pitch + 32 * V - 1) / (32 * V);
  const long item = (long)blockIdx.x * kWarpsX + threadIdx.y;
  const long nitems = ncs * ((ny + ROWS - 1) / ROWS);
  const long pc0 = ((item % ncs) * 32 + lane) * V;
  const bool live = item < nitems && pc0 < pitch;
  const int xl0 = (int)(pc0 - off);
  const int y0 = 1 + (int)(item / ncs) * ROWS;  // interior rows only
  // elements outside the logical array read as zero
  bool xin[V];
#pragma unroll
  for (int v = 0; v < V; ++v) xin[v] = xl0 + v >= 0 && xl0 + v <= nx + 1;
  auto load_u = [&](int y, T *o) {
    if (live && y <= ny + 1) {
      unpack<T, V>(*reinterpret_cast<const VT *>(u + (long)y * pitch + pc0), o);
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (!xin[v]) o[v] = T(0);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) o[v] = T(0);
    }
  };
  // rows streamed through a three-row window (y-1, y, y+1)
  T um[V], uc[V], up[V];
  load_u(y0 - 1, um);
  load_u(y0, uc);
  const bool lval = live && (xl0 - 1 >= 0) && (xl0 - 1 <= nx + 1);
  const bool rval = live && (xl0 + V <= nx + 1);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
  for (int r = 0; r < ROWS; ++r) {
    const int y = y0 + r;
    if (y > ny || item >= nitems) break;
    load_u(y + 1, up);
    T left = __shfl_up_sync(0xffffffffu, uc[V - 1], 1);
    T right = __shfl_down_sync(0xffffffffu, uc[0], 1);
    if (lane == 0) left = lval ? u[(long)y * pitch + pc0 - 1] : T(0);
    if (lane == 31) right = rval ? u[(long)y * pitch + pc0 + V] : T(0);
    T g[V];
    if (live) {
      unpack<T, V>(*reinterpret_cast<const VT *>(lam + (long)y * pitch + pc0), g);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) g[v] = T(0);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int x = xl0 + v;
      if (x < 1 || x > nx) continue;
      const double gv = (double)g[v];
      const double xm = (double)(v == 0 ? left : uc[v - 1]);
      const double xp = (double)(v == V - 1 ? right : uc[v + 1]);
      acc[0] = fma(gv, xm, acc[0]);
      acc[1] = fma(gv, xp, acc[1]);
      acc[2] = fma(gv, (double)um[v], acc[2]);
      acc[3] = fma(gv, (double)uc[v], acc[3]);
      acc[4] = fma(gv, (double)up[v], acc[4]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      um[v] = uc[v];
      uc[v] = up[v];
    }
  }
  block_partials(acc, partials);
}

// dw[d] += sum of the partials in a fixed order (one block).
__global__ void wgrad_final_kernel(const double *__restrict__ partials, long nblocks, double *__restrict__ dw) {
  __shared__ double red[256][5];
  double acc[5] = {0, 0, 0, 0, 0};
  for (long b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int d = 0; d < 5; ++d) acc[d] += partials[b * 5 + d];
  for (int d = 0; d < 5; ++d) red[threadIdx.x][d] = acc[d];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int d = 0; d < 5; ++d) red[threadIdx.x][d] += red[threadIdx.x + s][d];
    __syncthreads();
  }
  if (threadIdx.x < 5) dw[threadIdx.x] += red[0][threadIdx.x];
}

// FMA throughput probe: eight independent chains per thread.
template <typename T>
__global__ void fma_rate_kernel(T *out, int iters, T a, T b) {
  T r0 = threadIdx.x, r1 = r0 + 1, r2 = r0 + 2, r3 = r0 + 3, r4 = r0 + 4, r5 = r0 + 5, r6 = r0 + 6, r7 = r0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      r0 = fma_rn(r0, a, b); r1 = fma_rn(r1, a, b); r2 = fma_rn(r2, a, b); r3 = fma_rn(r3, a, b);
      r4 = fma_rn(r4, a, b); r5 = fma_rn(r5, a, b); r6 = fma_rn(r6, a, b); r7 = fma_rn(r7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = r0 + r1 + r2 + r3 + r4 + r5 + r6 + r7;
}

// Integer-path throughput probe: four independent cell evaluations per
// iteration, each on its own five inputs (a sliding window of its previous
// outputs), so nothing is hoisted out of the loop.  Weights sum to about 1
// and the inputs stay in (0, 1): every evaluation takes the fast path.
__global__ void exact_rate_kernel(double *out, int iters, ExactW u, Links<double> a) {
  double s[4][5];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 5; ++i) s[j][i] = 0.05 + 0.04 * (j * 5 + i) + threadIdx.x * 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double o = stencil_cell(a, u, true, s[j][0], s[j][1], s[j][2], s[j][3], s[j][4]);
#pragma unroll
      for (int i = 4; i > 0; --i) s[j][i] = s[j][i - 1];
      s[j][0] = o;
    }
  }
  double acc = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc += s[j][0];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The same probe for the 9-term integer path of the 3x3 box.
__global__ void exact_rate_box_kernel(double *out, int iters, ExactWN<9> u, Box9<double> b) {
  double s[2][9];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int i = 0; i < 9; ++i) s[j][i] = 0.05 + 0.03 * (j * 9 + i) + threadIdx.x * 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double o = stencil_box_cell(b, u, true, s[j][0], s[j][1], s[j][2], s[j][3], s[j][4], s[j][5], s[j][6],
                                        s[j][7], s[j][8]);
#pragma unroll
      for (int i = 8; i > 0; --i) s[j][i] = s[j][i - 1];
      s[j][0] = o;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s[0][0] + s[1][0];
}

// ---- host launchers --------------------------------------------------------

template <typename T>
static Weights<T> cast_weights(const double *w) {
  Weights<T> r;
  for (int i = 0; i < 5; ++i) r.w[i] = (T)w[i];
  return r;
}

constexpr int kOneRows = 8;       // rows per work item, FP64 (arithmetic bound: FP64 and integer pipes)
constexpr int kOneRowsF32 = 16;   // FP32 (HBM bound): more rows, fewer halo re-reads
constexpr int kWgradRows = 32;    // rows per thread of the weight gradient (streamed): amortises the reduction
constexpr int kOneRowsWG = 4;     // rows per work item of the fused adjoint step + weight gradient (registers)
constexpr int kBoxRows = 4;       // rows per work item of the one-step box kernel, FP64 (registers)
constexpr int kBoxRowsF32 = 8;    // the same, FP32

std::atomic<long> g_launches{0};

// Grid of the persistent one-step kernel: enough blocks for every work item,
// at most the number that fit on the device at once.
template <typename K>
static dim3 persistent_grid(K kernel, const GridDesc &g, int vec, int rows) {
  static thread_local int cached_dev = -1, cached_sms = 0;
  static thread_local const void *cached_k = nullptr;
  static thread_local int cached_blocks = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != cached_dev || (const void *)kernel != cached_k) {
    cudaDeviceGetAttribute(&cached_sms, cudaDevAttrMultiProcessorCount, dev);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 32 * kWarpsX, 0);
    cached_blocks = std::max(1, per) * cached_sms;
    cached_dev = dev;
    cached_k = (const void *)kernel;
  }
  const long ncs = (g.pitch + 32 * vec - 1) / (32 * vec);
  const long nitems = ncs * ((g.ny + 2 + rows - 1) / rows);
  const long need = (nitems + kWarpsX - 1) / kWarpsX;
  return dim3((unsigned)std::max<long>(1, std::min<long>(need, cached_blocks)));
}

cudaError_t launch_onestep(j2d_dtype dt, bool adj, const void *in, void *out, const GridDesc &g, int ipath,
                           cudaStream_t s) {
  note_launch();
  const dim3 blk(32, kWarpsX);
  if (g.shape == 9) {  // the 3x3 box: forward only
    if (dt == J2D_F64) {
      const dim3 grd = persistent_grid(onestep_box_kernel<double, kBoxRows>, g, 2, kBoxRows);
      onestep_box_kernel<double, kBoxRows><<<grd, blk, 0, s>>>((const double *)in, (double *)out, g.pitch,
                                                               (int)g.off, g.nx, g.ny, box_chain<double>(g.w), ipath);
    } else {
      const dim3 grd = persistent_grid(onestep_box_kernel<float, kBoxRowsF32>, g, 4, kBoxRowsF32);
      onestep_box_kernel<float, kBoxRowsF32><<<grd, blk, 0, s>>>((const float *)in, (float *)out, g.pitch,
                                                                 (int)g.off, g.nx, g.ny, box_chain<float>(g.w), 0);
    }
    return cudaGetLastError();
  }
  if (dt == J2D_F64) {
    const dim3 grd = adj ? persistent_grid(onestep_kernel<double, true, kOneRows>, g, 2, kOneRows)
                         : persistent_grid(onestep_kernel<double, false, kOneRows>, g, 2, kOneRows);
    auto w = cast_weights<double>(g.w);
    if (adj)
      onestep_kernel<double, true, kOneRows><<<grd, blk, 0, s>>>((const double *)in, (double *)out, g.pitch,
                                                                 (int)g.off, g.nx, g.ny, w, ipath);
    else
      onestep_kernel<double, false, kOneRows><<<grd, blk, 0, s>>>((const double *)in, (double *)out, g.pitch,
                                                                  (int)g.off, g.nx, g.ny, w, ipath);
  } else {
    const dim3 grd = adj ? persistent_grid(onestep_kernel<float, true, kOneRowsF32>, g, 4, kOneRowsF32)
                         : persistent_grid(onestep_kernel<float, false, kOneRowsF32>, g, 4, kOneRowsF32);
    auto w = cast_weights<float>(g.w);
    if (adj)
      onestep_kernel<float, true, kOneRowsF32><<<grd, blk, 0, s>>>((const float *)in, (float *)out, g.pitch,
                                                                (int)g.off, g.nx, g.ny, w, 0);
    else
      onestep_kernel<float, false, kOneRowsF32><<<grd, blk, 0, s>>>((const float *)in, (float *)out, g.pitch,
                                                                 (int)g.off, g.nx, g.ny, w, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_ring_copy(j2d_dtype dt, const void *in, void *out, const GridDesc &g, cudaStream_t s,
                             long count, long ostride) {
  const int n = 2 * (g.nx + 2) + 2 * g.ny;
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  const dim3 grd((unsigned)blocks, (unsigned)std::min<long>(std::max<long>(count, 1), 1024));
  note_launch();
  if (dt == J2D_F64)
    ring_copy_kernel<double><<<grd, 256, 0, s>>>((const double *)in, (double *)out, g.pitch, (int)g.off, g.nx, g.ny,
                                                 ostride, count);
  else
    ring_copy_kernel<float><<<grd, 256, 0, s>>>((const float *)in, (float *)out, g.pitch, (int)g.off, g.nx, g.ny,
                                                ostride, count);
  return cudaGetLastError();
}

long wgrad_partial_count(j2d_dtype dt, const GridDesc &g) {
  const int V = dt == J2D_F64 ? 2 : 4;
  const long ncs = (g.pitch + 32 * V - 1) / (32 * V);
  const long nitems = ncs * ((g.ny + kWgradRows - 1) / kWgradRows);
  return (nitems + kWarpsX - 1) / kWarpsX;
}

cudaError_t launch_wgrad(j2d_dtype dt, const void *u, const void *lam, double *dw, double *partials,
                         const GridDesc &g, cudaStream_t s) {
  const dim3 blk(32, kWarpsX);
  const dim3 grd((unsigned)wgrad_partial_count(dt, g));
  note_launch(2);
  if (dt == J2D_F64)
    wgrad_kernel<double, kWgradRows><<<grd, blk, 0, s>>>((const double *)u, (const double *)lam, g.pitch,
                                                         (int)g.off, g.nx, g.ny, partials);
  else
    wgrad_kernel<float, kWgradRows><<<grd, blk, 0, s>>>((const float *)u, (const float *)lam, g.pitch, (int)g.off,
                                                        g.nx, g.ny, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wgrad_final_kernel<<<1, 256, 0, s>>>(partials, (long)grd.x, dw);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_wgrad(j2d_dtype dt, const void *u, const void *lam1, void *lam0, double *dw,
                                 double *partials, long max_partials, const GridDesc &g, int ipath, cudaStream_t s) {
  note_launch(2);
  const dim3 blk(32, kWarpsX);
  if (dt == J2D_F64) {
    auto k = onestep_kernel<double, true, kOneRowsWG, true>;
    dim3 grd = persistent_grid(k, g, 2, kOneRowsWG);
    grd.x = (unsigned)std::max<long>(1, std::min<long>(grd.x, max_partials));
    k<<<grd, blk, 0, s>>>((const double *)lam1, (double *)lam0, g.pitch, (int)g.off, g.nx, g.ny,
                          cast_weights<double>(g.w), ipath, (const double *)u, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wgrad_final_kernel<<<1, 256, 0, s>>>(partials, (long)grd.x, dw);
  } else {
    auto k = onestep_kernel<float, true, kOneRowsWG, true>;
    dim3 grd = persistent_grid(k, g, 4, kOneRowsWG);
    grd.x = (unsigned)std::max<long>(1, std::min<long>(grd.x, max_partials));
    k<<<grd, blk, 0, s>>>((const float *)lam1, (float *)lam0, g.pitch, (int)g.off, g.nx, g.ny,
                          cast_weights<float>(g.w), 0, (const float *)u, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wgrad_final_kernel<<<1, 256, 0, s>>>(partials, (long)grd.x, dw);
  }
  return cudaGetLastError();
}

// Rows of a dense host array (device-accessible pinned memory) into the plan
// layout: one block per row at a time, four loads in flight per thread.  The
// loads cross the host link from many SMs at once; a DMA copy issued right
// after a long kernel measured 10-40 GB/s against about 200 for this gather.
template <typename T>
__global__ void __launch_bounds__(512) gather_rows_kernel(const T *__restrict__ src, long spitch, T *__restrict__ dst,
                                                           long dpitch, long rows, long width) {
  constexpr int U = 4;
  for (long r = blockIdx.x; r < rows; r += gridDim.x) {
    const T *s = src + r * spitch;
    T *d = dst + r * dpitch;
    for (long c0 = (long)threadIdx.x; c0 < width; c0 += (long)U * blockDim.x) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long c = c0 + (long)u * blockDim.x;
        if (c < width) v[u] = s[c];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long c = c0 + (long)u * blockDim.x;
        if (c < width) d[c] = v[u];
      }
    }
  }
}

cudaError_t launch_gather_rows(j2d_dtype dt, const void *src, long spitch, void *dst, long dpitch, long rows, long width,
                               cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const unsigned blocks = (unsigned)std::max<long>(1, std::min<long>(rows, (long)sms * 4));
  note_launch();
  if (dt == J2D_F64)
    gather_rows_kernel<double><<<blocks, 512, 0, s>>>((const double *)src, spitch, (double *)dst, dpitch, rows, width);
  else
    gather_rows_kernel<float><<<blocks, 512, 0, s>>>((const float *)src, spitch, (float *)dst, dpitch, rows, width);
  return cudaGetLastError();
}

cudaError_t measure_fma(j2d_dtype dt, double *rate) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blk = 256, grid = sms * 8;
  const int iters = dt == J2D_F64 ? 400 : 8000;
  void *buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(double) * grid * blk)) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (dt == J2D_F64)
      fma_rate_kernel<double><<<grid, blk>>>((double *)buf, iters, 0.999, 0.001);
    else
      fma_rate_kernel<float><<<grid, blk>>>((float *)buf, iters, 0.999f, 0.001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  *rate = (double)grid * blk * iters * 64 / (best * 1e-3);
  return cudaSuccess;
}

cudaError_t measure_exact(double *rate) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blk = 256, grid = sms * 8, iters = 200;
  void *buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(double) * grid * blk)) != cudaSuccess) return e;
  const Links<double> a{0.21, 0.19, 0.2, 0.18, 0.22};
  ExactW u;
  const double w[5] = {a.xm, a.xp, a.ym, a.c, a.yp};
  u.ok = true;
  for (int i = 0; i < 5; ++i) {
    uint64_t b;
    memcpy(&b, &w[i], 8);
    u.e[i] = (int)(b >> 52);
    u.m[i] = (b & ((1ull << 52) - 1)) | (1ull << 52);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    exact_rate_kernel<<<grid, blk>>>((double *)buf, iters, u, a);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  *rate = (double)grid * blk * iters * 4 / (best * 1e-3);
  return cudaSuccess;
}

cudaError_t measure_exact_box(double *rate) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blk = 256, grid = sms * 8, iters = 200;
  void *buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(double) * grid * blk)) != cudaSuccess) return e;
  const double w[9] = {0.11, 0.12, 0.1, 0.115, 0.105, 0.11, 0.1, 0.12, 0.11};  // positive, summing to 1
  const Box9<double> b = box_chain<double>(w);
  ExactWN<9> u;
  u.ok = true;
  for (int i = 0; i < 9; ++i) {
    uint64_t bits;
    memcpy(&bits, &b.w[i], 8);
    u.e[i] = (int)(bits >> 52);
    u.m[i] = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    exact_rate_box_kernel<<<grid, blk>>>((double *)buf, iters, u, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  *rate = (double)grid * blk * iters * 2 / (best * 1e-3);
  return cudaSuccess;
}

// Shared-memory bandwidth probe: each thread owns 8 16-byte slots of a 64 KB
// buffer (lane-consecutive, bank-conflict free, the access pattern of the
// strip sweeps) and per step loads one slot and stores it to another of its
// own, so threads never share an address.
__global__ void __launch_bounds__(512) smem_rate_kernel(float *out, int iters) {
  extern __shared__ float4 sbuf[];  // 8 * blockDim.x float4
  const int t = threadIdx.x, nb = blockDim.x;
#pragma unroll
  for (int k = 0; k < 8; ++k) sbuf[t + k * nb] = make_float4((float)(t + k), 0.f, 0.f, 0.f);
  __syncwarp();
  // volatile accesses: the compiler may not forward a thread's own stores to
  // its later loads through registers
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(sbuf);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float4 v;
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "r"(base + (uint32_t)(t + k * nb) * 16u));
      acc.x += v.x;
      asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(base + (uint32_t)(t + ((k + 4) & 7) * nb) * 16u),
                   "f"(v.y), "f"(v.z), "f"(v.w), "f"(v.x + 1.f)
                   : "memory");
    }
  }
  out[blockIdx.x * nb + t] = acc.x + acc.y + acc.z + acc.w;
}

cudaError_t measure_smem(double *bytes_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blk = 512, grid = sms * 2, iters = 2000;
  const size_t smem = (size_t)8 * blk * sizeof(float4);  // 64 KB
  if ((e = cudaFuncSetAttribute(smem_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  void *buf = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(float) * grid * blk)) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    smem_rate_kernel<<<grid, blk, smem>>>((float *)buf, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  // 8 loads and 8 stores of 16 bytes per thread per iteration
  *bytes_per_s = (double)grid * blk * iters * 8 * 2 * 16 / (best * 1e-3);
  return cudaSuccess;
}

}  // namespace j2d
