// dtb.cu -- deep temporal blocking (DTB) kernels for j2d5pt on sm_103a.
//
// The method (Zhang et al., GPGPU'23, Sections 3.1-3.3, Figure 1): tile the
// domain so that a tile fills the GPU's shared memory, load it once, advance
// it several time steps on chip with device-wide synchronisation resolving
// the halos between thread blocks, then store it; tiles are processed one
// after another.  The paper's step function (Listing 1) is the same whether
// its pointers address global or shared memory.
//
// GB300 design.  The unit of work is a warp-owned *strip*: 32 lanes x one
// 16-byte vector each (64 FP64 or 128 FP32 columns) by up to R rows, held in
// the CTA's shared memory.  A warp sweeps its strip row by row with a
// three-row register window (the listing's column cache), exchanges the x+-1
// neighbours across lanes with shuffles, and updates the strip in place.
// Halos between strips are point to point: at the end of every step a strip
// writes its four edges into double-buffered mailboxes of its neighbours
// (shared memory when the neighbour is in the same CTA, L2-resident global
// memory otherwise) and publishes a per-warp step counter; a strip waits only
// for its own (at most four) neighbours' counters (FP32 strips of one CTA use
// one CTA barrier per step instead, faster for their short steps).  This
// replaces the paper's grid-wide barrier per step with neighbour
// synchronisation that never stalls unrelated CTAs.  Strips are loaded with 2D TMA tensor copies and written
// back with per-row TMA tensor stores (the store tensor map ends at the last
// interior row/column, so the ring and padding are never written).
//
// Four schedules drive the same strip code:
//   RESIDENT  all strips of the grid on chip at once, every step exchanged
//             (the grid must fit in the GPU's shared memory);
//   BANDS     the paper's serial GPU-wide tiles: full-width bands of rows
//             with a k-row overlapped halo above and below, k steps per visit;
//   TILES     independent CTA tiles with a k-deep overlapped halo on all sides
//             (no cross-CTA exchange at all), k steps per visit; also carries
//             batches of grids, partial tiles packed side by side in a CTA;
//   SKEWED    serial tiles in skewed coordinates: each CTA advances a run of
//             rows of a column band tile after tile, each tile taking its top
//             halo at every step from the tile before it, so no halo is
//             recomputed in y (run_strip_skew).
// RESIDENT on a batch runs the grids in waves (MODE_GROUPS): the grids of a
// wave are on chip together, each split into strips whose links stay inside
// it, advanced all steps with the neighbour exchange, and stored; a grid
// barrier separates the waves.
// In RESIDENT and BANDS a CTA holds a block of strips (4 x 4 where the grid
// allows; see choose_bx), so that most neighbours share its shared memory.
// FP32 TILES strips take two steps per exchange (run_strip_pair), reading
// their neighbours' cells in place.
// Every wait is bounded by a %globaltimer deadline; on expiry the kernel
// records J2D_ERR_TIMEOUT, stops waiting and runs to completion.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <functional>
#include <queue>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "dtb.h"

namespace j2d {

constexpr int kWarps = 16;            // warps (strips) per CTA
constexpr int kThreads = kWarps * 32;
enum { SIDE_YM = 0, SIDE_YP = 1, SIDE_XM = 2, SIDE_XP = 3 };
enum { LINK_CONST = -1, LINK_ZERO = -2 };
enum { MODE_BANDS = 0, MODE_TILES = 1, MODE_TILES_PAIR = 2, MODE_SKEW = 3, MODE_GROUPS = 4 };
// A tile job: grid, tile origin (x, y), valid core [vx0, vx1) x [vy0, vy1),
// first warp, strips across and down (only the strips inside the grid: a
// CTA runs a group of partial tiles side by side), and in the first tile of
// a group the number of tiles in the group (so that a group is read with its
// first record, no extra indirection).
constexpr int kTileInts = 11;
// A skewed tile job (SKEWED schedule): grid, band origin tx0 and valid
// columns [vx0, vx1), first skewed row q0 and row count nq of the tile, the
// physical rows [v0, v1) of the tile's piece whose values the tile stores
// (skewed rows [v0+k, v1+k) at level k), first = 1 when the tile opens a
// piece (no predecessor in the CTA's list), and wxa, the strips across
// inside the grid.
constexpr int kSkewInts = 10;
// A strip of a grouped-resident wave (RESIDENT for a batch), one record per
// slot (CTA x 16 + warp) and wave: grid (-1: no strip), first cell (x0, y0),
// rows, ring bits, and the four neighbour slots (SIDE_* order) or LINK_CONST.
constexpr int kSlotInts = 9;

// Per-grid data the kernel reads from global memory.
struct GridDev {
  int nx, ny, off, shape;
  long pitch;
  double w[9];  // {W, E, S, C, N}, or the nine box weights in row order
  void *buf[3];  // 0 = in, 1 = workspace, 2 = out
};

struct KParams {
  const GridDev *grids;
  const CUtensorMap *maps;  // per grid: load maps of buf[0..2], store maps of buf[0..2]
  const int *jobs;          // BANDS: 5 ints per wave; TILES: kTileInts ints per tile
  const int *job_off;       // TILES: CTA b processes tiles [job_off[b], job_off[b+1]), group by group
  int njobs;                // waves (BANDS) or tiles (TILES) per round
  int rounds, depth, last_depth, src0;
  int rmax, rp;             // strip rows (max), mailbox column length
  int m;                    // BANDS: strips per column (per-wave value in the job)
  int bx;                   // BANDS: CTA block of bx x (16/bx) strips, 0 = 16 strips down a column
  int tile_rows;            // TILES: rows per strip (tile shapes are per job)
  int *status;
  int *barrier;             // grid barrier counter
  int *gflags;              // per slot step counters (cross-CTA consumers)
  void *gslots;             // per slot mailboxes (cross-CTA consumers)
  unsigned long long timeout_ns;
  int mute_slot;            // fault injection: this slot never publishes its step counter (-1: none)
  int int_path;             // FP64: the kExactMask cells on the integer path
  unsigned long long mem_lo, mem_hi;  // checked build: the global range this launch may touch
  void *skewbuf;            // SKEWED: per CTA [2 parities][levels][2 rows][skew_tw] elements
  int skew_tw, skew_levels, skew_wx;  // SKEWED: band width (elements), levels per parity, strips across
  int dead_all;             // RESIDENT / BANDS, FP64: some strip has dead columns, all take the dead-column sweep
  void *states;             // forward runs keeping every state: state t+1 at states + t * state_elems (or null)
  long state_elems;
};

// Layout of one warp's shared-memory region (elements of T).
template <typename T>
struct WarpLayout {
  static constexpr int V = VecOf<T>::V;
  static constexpr int SW = 32 * V;
  __host__ __device__ static int mailbox_elems(int rp) { return 4 * SW + 4 * rp; }
  __host__ __device__ static int region_elems(int rmax, int rp) {
    const int e = rmax * SW + mailbox_elems(rp);
    const int per128 = 128 / (int)sizeof(T);
    return (e + per128 - 1) / per128 * per128;
  }
  // offsets of the mailboxes inside a mailbox block: ym[2][SW], yp[2][SW], xm[2][rp], xp[2][rp]
  __host__ __device__ static int side_off(int side, int rp) {
    return side == SIDE_YM ? 0 : side == SIDE_YP ? 2 * SW : side == SIDE_XM ? 4 * SW : 4 * SW + 2 * rp;
  }
  __host__ __device__ static int side_len(int side, int rp) { return side <= SIDE_YP ? SW : rp; }
};

constexpr int kHeaderBytes = 1024;  // mbarriers and step counters at the start of shared memory

__host__ __device__ inline size_t dtb_smem_bytes(int elem, int rmax, int rp) {
  const int SW = 32 * (16 / elem);
  int e = rmax * SW + 4 * SW + 4 * rp;
  const int per128 = 128 / elem;
  e = (e + per128 - 1) / per128 * per128;
  return (size_t)kHeaderBytes + (size_t)kWarps * e * elem;
}

// Two-steps-per-sweep tiles (FP32 forward): a warp's region is its strip and
// four 32-entry halo columns (columns -1 and SW at step t, then at step t+1),
// with no mailboxes: neighbours' cells are read in place.
constexpr int kPairCols = 4 * 32;
__host__ __device__ inline int pair_region_elems(int elem, int rmax) {
  const int SW = 32 * (16 / elem);
  const int per128 = 128 / elem;
  return (rmax * SW + kPairCols + per128 - 1) / per128 * per128;
}
__host__ __device__ inline size_t pair_smem_bytes(int elem, int rmax) {
  return (size_t)kHeaderBytes + (size_t)kWarps * pair_region_elems(elem, rmax) * elem;
}

// ---- memory accessors (tested in the checked build) --------------------------

#ifdef J2D_BOUNDS_CHECK
__device__ int g_bounds_fault;                       // J2D_ERR_BOUNDS once a test failed
__shared__ unsigned long long s_mem_lo, s_mem_hi;    // global range the launch may touch
#endif

// Is [p, p + bytes) inside the launch's shared memory (shared addresses) or
// inside the launch's global range?  Always true in the regular build.
__device__ __forceinline__ bool access_ok(const void *p, unsigned bytes) {
#ifdef J2D_BOUNDS_CHECK
  bool ok;
  if (__isShared(p)) {
    ok = smem_window_ok(p, bytes);
  } else {
    const unsigned long long a = (unsigned long long)p;
    ok = a >= s_mem_lo && a + bytes <= s_mem_hi;
  }
  if (!ok) atomicCAS(&g_bounds_fault, DEV_OK, DEV_BOUNDS);
  return ok;
#else
  (void)p;
  (void)bytes;
  return true;
#endif
}
template <typename T> __device__ __forceinline__ T ldm(const T *p) {
  if (kChecked && !access_ok(p, sizeof(T))) return T(0);
  return *p;
}
template <typename T> __device__ __forceinline__ void stm(T *p, T v) {
  if (!kChecked || access_ok(p, sizeof(T))) *p = v;
}
template <typename T> __device__ __forceinline__ T ld_cg_chk(const T *p) {
  if (kChecked && !access_ok(p, sizeof(T))) return T(0);
  return ld_cg(p);
}

// ---- bounded waits ---------------------------------------------------------

__device__ __forceinline__ bool expired(uint64_t deadline, int *status) {
  if (has_error(status)) return true;
  if (globaltimer_ns() > deadline) {
    set_error(status, DEV_TIMEOUT);
    return true;
  }
  return false;
}

// All lanes wait until *flag >= target (acquire); false on timeout / error.
__device__ __forceinline__ bool wait_flag(const int *flag, bool global, int target, const KParams &kp) {
  if (kChecked && !access_ok(flag, 4)) return false;
  const uint64_t deadline = globaltimer_ns() + kp.timeout_ns;
  for (int it = 0;; ++it) {
    const int v = global ? ld_acquire_gpu(flag) : ld_acquire_cta(flag);
    if (__all_sync(0xffffffffu, v >= target)) return true;
    if ((it & 63) == 63) {
      if (__any_sync(0xffffffffu, expired(deadline, kp.status))) return false;
      if (global) __nanosleep(64);
    }
  }
}

__device__ __forceinline__ bool wait_mbar(uint64_t *bar, uint32_t parity, const KParams &kp) {
  const uint64_t deadline = globaltimer_ns() + kp.timeout_ns;
  for (int it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15) == 15 && expired(deadline, kp.status)) return false;
  }
}

__device__ void grid_barrier(const KParams &kp, int &epoch) {
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    fence_acq_rel_gpu();
    atomicAdd(kp.barrier, 1);
    const int target = epoch * (int)gridDim.x;
    const uint64_t deadline = globaltimer_ns() + kp.timeout_ns;
    while (ld_acquire_gpu(kp.barrier) < target) {
      if (expired(deadline, kp.status)) break;
      __nanosleep(128);
    }
  }
  __syncthreads();
}

// ---- strips ----------------------------------------------------------------

// A strip's next load, prefetched into L2 while the current strip runs.
struct Prefetch {
  const CUtensorMap *map = nullptr;  // none when null
  int x = 0, y = 0;
};

struct Strip {
  int g;              // grid index
  int x0, y0, rows;   // logical coordinates of the first cell; number of rows
  int link[4];        // neighbour slot (>= 0), LINK_CONST or LINK_ZERO
  int ring;           // bit per side: that side is the domain ring
  int sy0, sy1;       // rows to store (strip-relative)
  int sx0, sx1;       // columns to store (strip-relative)
  int tw;             // TILES: strips across the strip's tile
  bool active;
};

template <typename T>
__device__ __forceinline__ void vload(const T *p, bool global, T *o) {
  if (kChecked && !access_ok(p, 16)) {
    for (int e = 0; e < 16 / (int)sizeof(T); ++e) o[e] = T(0);
    return;
  }
  if constexpr (sizeof(T) == 8) {
    double2 v = global ? __ldcg(reinterpret_cast<const double2 *>(p)) : *reinterpret_cast<const double2 *>(p);
    o[0] = v.x; o[1] = v.y;
  } else {
    float4 v = global ? __ldcg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
}
template <typename T>
__device__ __forceinline__ void vstore(T *p, const T *o) {
  if (kChecked && !access_ok(p, 16)) return;
  if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
  } else {
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

// Adjoint ring accumulators of a strip bordering the ring (unused forward).
template <typename T>
struct RingAcc {
  T ym[VecOf<T>::V], yp[VecOf<T>::V];  // ring rows 0 and ny+1, this lane's columns
  T xm0, xm1, xp0, xp1;                // ring columns 0 and nx+1, rows lane and lane+32
  int ring, xp_lane, xp_elem;
  T W, E, S, N;
};

// Dead cells (strip columns beyond the grid) of FP64 sweeps are skipped
// rather than evaluated and discarded (see sweep_row).
template <typename T> constexpr bool kSkipDead = sizeof(T) == 8;

// One row r of a strip sweep: new values of row r from the old rows r-1 (ra),
// r (rb) and r+1 (rc), stored in place, then the window moves down a row.
template <typename T, bool ADJ, bool DEAD>
__device__ __forceinline__ void sweep_row(T (&ra)[VecOf<T>::V], T (&rb)[VecOf<T>::V], const T (&rc)[VecOf<T>::V],
                                          T *drow, const T *hcol, int r, int rows, int lane, const Links<T> &a,
                                          const ExactW &u, bool ipath, int xl, int y0, uint32_t dead,
                                          RingAcc<T> &rg) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  const T h = ldm(&hcol[r]);
  T left = __shfl_up_sync(0xffffffffu, rb[V - 1], 1);
  T right = __shfl_down_sync(0xffffffffu, rb[0], 1);
  if (lane == 0) left = h;
  if (lane == 31) right = h;
  T o[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    // an FP64 dead cell keeps its value and is not evaluated (its zero-filled
    // neighbours would send it off the integer path onto the FMA chain); FP32
    // selects after evaluating (skipping measured slower there)
    if (kSkipDead<T> && DEAD && (dead & (1u << e))) {
      o[e] = rb[e];
      continue;
    }
    const T xm = e == 0 ? left : rb[e - 1], xp = e == V - 1 ? right : rb[e + 1];
    if constexpr (std::is_same<T, double>::value)
      o[e] = stencil_cell(a, u, exact_cell(xl + e, y0 + r, ipath), xm, xp, ra[e], rb[e], rc[e]);
    else
      o[e] = stencil(a, xm, xp, ra[e], rb[e], rc[e]);
  }
  if constexpr (!kSkipDead<T> && DEAD) {
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (dead & (1u << e)) o[e] = rb[e];
  }
  vstore(drow + r * SW, o);
#pragma unroll
  for (int e = 0; e < V; ++e) { ra[e] = rb[e]; rb[e] = rc[e]; }
}

// One time step over a strip held in shared memory, swept row by row with a
// three-row register window and updated in place.  Only this warp's own
// shared memory is touched: the halo rows come in registers, the halo column
// from the warp's mailbox (lane 0 reads the x-1 column, lane 31 the x+1 one).
template <typename T, bool ADJ, bool DEAD>
__device__ __forceinline__ void sweep_rows(T *drow, const T *hcol, int rows, int lane, const Links<T> &a,
                                           const ExactW &u, bool ipath, int xl, int y0, const T *hym,
                                           const T *hyp, uint32_t dead, RingAcc<T> &rg) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  T ra[V], rb[V], rc[V];
#pragma unroll
  for (int e = 0; e < V; ++e) ra[e] = hym[e];
  vload(drow, false, rb);
  // FP32: unrolling by the window's period (3) lets the compiler rename the
  // three row registers instead of moving them (measured +9%); FP64 prefers 2
  // FP32 peels the last row so the loop loads the next row unconditionally
  // (+3-4%); FP64 keeps one loop (peeling measured -7% there)
  constexpr int kUnroll = sizeof(T) == 4 ? 3 : 2;
  if constexpr (sizeof(T) == 4) {
#pragma unroll kUnroll
    for (int r = 0; r < rows - 1; ++r) {
      vload(drow + (r + 1) * SW, false, rc);
      sweep_row<T, ADJ, DEAD>(ra, rb, rc, drow, hcol, r, rows, lane, a, u, ipath, xl, y0, dead, rg);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) rc[e] = hyp[e];
    sweep_row<T, ADJ, DEAD>(ra, rb, rc, drow, hcol, rows - 1, rows, lane, a, u, ipath, xl, y0, dead, rg);
  } else {
#pragma unroll kUnroll
    for (int r = 0; r < rows; ++r) {
      if (r + 1 < rows) {
        vload(drow + (r + 1) * SW, false, rc);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) rc[e] = hyp[e];
      }
      sweep_row<T, ADJ, DEAD>(ra, rb, rc, drow, hcol, r, rows, lane, a, u, ipath, xl, y0, dead, rg);
    }
  }
}

// Adjoint ring cells of a strip bordering the ring, once per step and before
// the sweep overwrites the strip: each adds its link weight times the old
// value of its one interior neighbour, rounded as stencil() rounds a ring
// cell's chain (the row-0, column-0 and column nx+1 cells add it in one fused
// multiply-add after the centre term; the row ny+1 cell rounds the product
// first).  Lane r keeps the column rings of row r (and r+32).
template <typename T>
__device__ __forceinline__ void ring_accumulate(RingAcc<T> &rg, const T *data, const T *drow, int rows, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  if (rg.ring & (1 << SIDE_YM)) {
    T v[V];
    vload(drow, false, v);
#pragma unroll
    for (int e = 0; e < V; ++e) rg.ym[e] = fma_rn(rg.S, v[e], rg.ym[e]);
  }
  if (rg.ring & (1 << SIDE_YP)) {
    T v[V];
    vload(drow + (rows - 1) * SW, false, v);
#pragma unroll
    for (int e = 0; e < V; ++e) rg.yp[e] = add_rn(rg.yp[e], mul_rn(rg.N, v[e]));
  }
  if (rg.ring & (1 << SIDE_XM)) {
    if (lane < rows) rg.xm0 = fma_rn(rg.W, ldm(&data[lane * SW]), rg.xm0);
    if (lane + 32 < rows) rg.xm1 = fma_rn(rg.W, ldm(&data[(lane + 32) * SW]), rg.xm1);
  }
  if (rg.ring & (1 << SIDE_XP)) {
    const int c = rg.xp_lane * V + rg.xp_elem;  // strip column of grid column nx
    if (lane < rows) rg.xp0 = fma_rn(rg.E, ldm(&data[lane * SW + c]), rg.xp0);
    if (lane + 32 < rows) rg.xp1 = fma_rn(rg.E, ldm(&data[(lane + 32) * SW + c]), rg.xp1);
  }
}

// Write back the valid part of a strip: whole rows by TMA tensor stores when
// the strip's columns are all valid (the store map clips beyond column nx),
// else element by element; adjoint strips bordering the ring also write their
// ring accumulators.
template <typename T, bool ADJ>
__device__ void strip_store(const Strip &st, const GridDev &gd, const T *data, const CUtensorMap *map_store,
                            T *dstbuf, int lane, const RingAcc<T> &rg) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  const int nx = gd.nx, ny = gd.ny, rows = st.rows;
  const long pitch = gd.pitch;
  const int off = gd.off;
  const bool full = st.sx0 == 0 && st.sx1 == SW;
  if (full) {
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      for (int r = st.sy0; r < st.sy1; ++r)
        if (!kChecked || access_ok(data + r * SW, SW * sizeof(T))) tma_store_2d(map_store, off + st.x0, st.y0 + r, data + r * SW);
      bulk_commit();
      // a tensor store may rewrite the rest of the 16-byte granule holding
      // column nx, i.e. the ring cell nx+1: let it land before the adjoint
      // writes the ring below
      if (ADJ && (st.ring & (1 << SIDE_XP))) {
        bulk_wait_all();
        fence_proxy_async_all();
      }
    }
    __syncwarp();
  } else {
    for (int r = st.sy0; r < st.sy1; ++r) {
      const long rowoff = (long)(st.y0 + r) * pitch + off;
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int c = lane * V + e;
        if (c >= st.sx0 && c < st.sx1) stm(&dstbuf[rowoff + st.x0 + c], ldm(&data[r * SW + c]));
      }
    }
  }
  if (ADJ && st.ring) {
    // ring cells of the valid region
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int c = lane * V + e, x = st.x0 + c;
      const bool xin = x >= 1 && x <= nx && c >= st.sx0 && c < st.sx1;
      if ((st.ring & (1 << SIDE_YM)) && xin && st.sy0 == 0) stm(&dstbuf[off + x], rg.ym[e]);
      if ((st.ring & (1 << SIDE_YP)) && xin && st.sy1 == rows) stm(&dstbuf[(long)(ny + 1) * pitch + off + x], rg.yp[e]);
    }
    if ((st.ring & (1 << SIDE_XM)) && st.sx0 == 0) {
      if (lane < rows && lane >= st.sy0 && lane < st.sy1) stm(&dstbuf[(long)(st.y0 + lane) * pitch + off], rg.xm0);
      if (lane + 32 < rows && lane + 32 >= st.sy0 && lane + 32 < st.sy1)
        stm(&dstbuf[(long)(st.y0 + lane + 32) * pitch + off], rg.xm1);
    }
    if ((st.ring & (1 << SIDE_XP)) && (nx - st.x0) < st.sx1) {
      if (lane < rows && lane >= st.sy0 && lane < st.sy1)
        stm(&dstbuf[(long)(st.y0 + lane) * pitch + off + nx + 1], rg.xp0);
      if (lane + 32 < rows && lane + 32 >= st.sy0 && lane + 32 < st.sy1)
        stm(&dstbuf[(long)(st.y0 + lane + 32) * pitch + off + nx + 1], rg.xp1);
    }
  }
}

// Advance one strip by k steps: load, exchange, sweep, store.  Called by
// every warp of the CTA with the same k (inactive strips only take part in
// the per-step CTA barrier).  Exchange protocol: the four edge mailboxes of a
// strip are double-buffered by step parity; in step t a strip reads parity
// t&1 and writes its new edges into its neighbours' parity (t+1)&1.  A
// neighbour is ordered by its published step counter (release/acquire, at
// CTA scope in shared memory for FP64 neighbours in the same CTA, at GPU
// scope for a neighbour in another CTA), waited for only by the strips that
// border it; for FP32, neighbours in the same CTA are ordered by one CTA
// barrier per step instead.
// The valid cells of a strip (its rows [sy0, sy1) and columns [sx0, sx1)
// inside the grid) into the grid-shaped buffer `out`: a 16-byte store per
// lane and row where the lane's whole vector is valid, single elements where
// it is not.  Used for the intermediate states of a state-keeping run.
template <typename T>
__device__ void strip_store_plain(const Strip &st, const GridDev &gd, const T *drow, int lane, T *out) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  const int c0 = lane * V, xe = gd.nx - st.x0;  // last valid strip column
  const bool whole = c0 >= st.sx0 && c0 + V <= st.sx1 && c0 + V - 1 <= xe;
  for (int r = st.sy0; r < st.sy1; ++r) {
    T *row = out + (long)(st.y0 + r) * gd.pitch + gd.off + st.x0;
    if (whole) {
      T v[V];
      vload(drow + r * SW, false, v);
      vstore(row + c0, v);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int c = c0 + e;
        if (c >= st.sx0 && c < st.sx1 && c <= xe) stm(&row[c], ldm(&drow[r * SW + e]));
      }
    }
  }
}

template <typename T, bool ADJ>
__device__ void run_strip(const Strip &st, const KParams &kp, char *smem, int warp, int slot, int src, int dst,
                          int k, int base, uint32_t &mbar_phase, const Prefetch &pf = Prefetch{}, int step0 = 0) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  using L = WarpLayout<T>;
  const int lane = threadIdx.x & 31;
  const int rp = kp.rp;
  const int region = L::region_elems(kp.rmax, rp);
  T *wbase = reinterpret_cast<T *>(smem + kHeaderBytes);
  T *data = wbase + (size_t)warp * region;
  T *mbox = data + (size_t)kp.rmax * SW;  // my shared-memory mailboxes
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  const bool act = st.active;
  const GridDev &gd = kp.grids[act ? st.g : 0];
  const int nx = gd.nx, ny = gd.ny, rows = st.rows;
  const long pitch = gd.pitch;
  const int off = gd.off;
  const T *srcbuf = reinterpret_cast<const T *>(gd.buf[src]);
  T *dstbuf = reinterpret_cast<T *>(gd.buf[dst]);
  const CUtensorMap *map_load = kp.maps + (size_t)st.g * 6 + src;
  const CUtensorMap *map_store = kp.maps + (size_t)st.g * 6 + 3 + dst;
  const int NW = kWarps;
  const size_t slot_elems = (size_t)L::mailbox_elems(rp);
  T *gslots = reinterpret_cast<T *>(kp.gslots);

  // base weights W, E, S, C, N and the links of interior cells
  const T W = (T)gd.w[0], E = (T)gd.w[1], S = (T)gd.w[2], C = (T)gd.w[3], N = (T)gd.w[4];
  const Links<T> a = ADJ ? Links<T>{E, W, N, C, S} : Links<T>{W, E, S, C, N};
  ExactW u{};
  if constexpr (std::is_same<T, double>::value) u = exact_weights(a);

  // where my incoming halos live (per side) and where my outgoing edges go
  bool remote[4], any_remote = false;
  const T *inbox[4];
  T *outbox[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int n = act ? st.link[s] : LINK_ZERO;
    remote[s] = n >= 0 && (n / NW) != (slot / NW);
    any_remote |= remote[s];
    inbox[s] = remote[s] ? gslots + (size_t)slot * slot_elems + L::side_off(s, rp) : mbox + L::side_off(s, rp);
    const int opp = s ^ 1;
    outbox[s] = n < 0 ? nullptr
                      : remote[s] ? gslots + (size_t)n * slot_elems + L::side_off(opp, rp)
                                  : wbase + (size_t)(n % NW) * region + (size_t)kp.rmax * SW + L::side_off(opp, rp);
  }
  // Neighbours in the same CTA: FP64 strips use the step-counter protocol of
  // the cross-CTA links (in shared memory), so a warp waits only for its own
  // neighbours; FP32 strips, whose steps are short, use one CTA barrier per
  // step (each measured faster for its type).
  constexpr bool kLocalFlags = sizeof(T) == 8;
  int *sflags = reinterpret_cast<int *>(smem + 512);
  bool local[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) local[s] = act && st.link[s] >= 0 && !remote[s];
  auto publish_local = [&](int value) {
    if constexpr (kLocalFlags) {
      fence_acq_rel_cta();
      __syncwarp();
      if (lane == 0 && (!kChecked || access_ok(sflags + warp, 4))) st_relaxed_cta(sflags + warp, value);
      __syncwarp();
    }
  };
  auto publish_remote = [&](int value) {
    if (!any_remote) return;
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0 && slot != kp.mute_slot && (!kChecked || access_ok(kp.gflags + slot, 4)))
      st_relaxed_gpu(kp.gflags + slot, value);
    __syncwarp();
  };

  const int xl = st.x0 + lane * V;  // logical x of this lane's element 0
  T *drow = data + lane * V;        // this lane's vector in strip row 0
  // columns beyond nx are dead: they keep their value (the ring column nx+1
  // is read by column nx: the ring value forward, zero in the adjoint)
  uint32_t dead = 0;
#pragma unroll
  for (int e = 0; e < V; ++e)
    if (act && xl + e > nx) dead |= 1u << e;
  // adjoint ring accumulators; the element holding column nx feeds the right ring
  RingAcc<T> rg;
#pragma unroll
  for (int e = 0; e < V; ++e) { rg.ym[e] = T(0); rg.yp[e] = T(0); }
  rg.xm0 = rg.xm1 = rg.xp0 = rg.xp1 = T(0);
  rg.ring = ADJ && act ? st.ring : 0;
  rg.xp_lane = (nx - st.x0) / V;
  rg.xp_elem = (nx - st.x0) % V;
  rg.W = W; rg.E = E; rg.S = S; rg.N = N;
  // copy this strip's current edges into the neighbours' mailboxes of parity `par`
  auto publish_edges = [&](int par) {
    if (outbox[SIDE_YM]) {
      T o[V];
      vload(drow, false, o);
      vstore(outbox[SIDE_YM] + par * SW + lane * V, o);
    }
    if (outbox[SIDE_YP]) {
      T o[V];
      vload(drow + (rows - 1) * SW, false, o);
      vstore(outbox[SIDE_YP] + par * SW + lane * V, o);
    }
    if (outbox[SIDE_XM])
      for (int r = lane; r < rows; r += 32) stm(&outbox[SIDE_XM][par * rp + r], ldm(&data[r * SW]));
    if (outbox[SIDE_XP])
      for (int r = lane; r < rows; r += 32) stm(&outbox[SIDE_XP][par * rp + r], ldm(&data[r * SW + SW - 1]));
  };

  if (act) {
    // ---- load the strip (TMA) ----
    fence_proxy_async_all();  // earlier generic writes before the async-proxy load
    __syncwarp();
    if (lane == 0) {
      bulk_wait_read_all();  // previous strip's stores have read shared memory
      const uint32_t bytes = (uint32_t)(SW * kp.rmax * sizeof(T));
      const bool ok = !kChecked || access_ok(data, bytes);  // a refused load still completes the phase
      mbar_expect_tx(&bars[warp], ok ? bytes : 0u);
      if (ok) tma_load_2d(data, map_load, off + st.x0, st.y0, &bars[warp]);
    }
    // constant halos (ring in the forward map, overlapped-halo edge rows/columns)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (st.link[s] >= 0) continue;
      // the adjoint never reads ring cells (their links to the interior are removed)
      const bool zero = st.link[s] == LINK_ZERO || (ADJ && ((st.ring >> s) & 1));
      T *box = mbox + L::side_off(s, rp);
      const int len = L::side_len(s, rp);
      if (s <= SIDE_YP) {
        const int y = s == SIDE_YM ? st.y0 - 1 : st.y0 + rows;
        T v[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          const int x = xl + e;
          v[e] = (!zero && x >= 0 && x <= nx + 1 && y >= 0 && y <= ny + 1) ? ldm(&srcbuf[(long)y * pitch + off + x]) : T(0);
        }
        vstore(box + lane * V, v);
        vstore(box + len + lane * V, v);
      } else {
        const int x = s == SIDE_XM ? st.x0 - 1 : st.x0 + SW;
        for (int r = lane; r < rows; r += 32) {
          const int y = st.y0 + r;
          const T v = (!zero && x >= 0 && x <= nx + 1) ? ldm(&srcbuf[(long)y * pitch + off + x]) : T(0);
          stm(&box[r], v);
          stm(&box[len + r], v);
        }
      }
    }
    // adjoint ring accumulators start from the ring values of the source
    if (ADJ) {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int x = xl + e;
        const bool xin = x >= 1 && x <= nx;
        if ((st.ring & (1 << SIDE_YM)) && xin) rg.ym[e] = ldm(&srcbuf[off + x]);
        if ((st.ring & (1 << SIDE_YP)) && xin) rg.yp[e] = ldm(&srcbuf[(long)(ny + 1) * pitch + off + x]);
      }
      if (st.ring & (1 << SIDE_XM)) {
        if (lane < rows) rg.xm0 = ldm(&srcbuf[(long)(st.y0 + lane) * pitch + off]);
        if (lane + 32 < rows) rg.xm1 = ldm(&srcbuf[(long)(st.y0 + lane + 32) * pitch + off]);
      }
      if (st.ring & (1 << SIDE_XP)) {
        if (lane < rows) rg.xp0 = ldm(&srcbuf[(long)(st.y0 + lane) * pitch + off + nx + 1]);
        if (lane + 32 < rows) rg.xp1 = ldm(&srcbuf[(long)(st.y0 + lane + 32) * pitch + off + nx + 1]);
      }
    }
    wait_mbar(&bars[warp], mbar_phase, kp);
    mbar_phase ^= 1u;
    if (pf.map && lane == 0) tma_prefetch_2d(pf.map, pf.x, pf.y);
    if (ADJ && dead) {
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (xl + e == nx + 1)
          for (int r = 0; r < rows; ++r) stm(&drow[r * SW + e], T(0));
    }
    __syncwarp();
    // ---- publish state-0 edges into the neighbours' parity-0 mailboxes ----
    publish_edges(0);
    publish_local(base);
    publish_remote(base);
  }
  __syncthreads();

  // ---- k steps ----
  // lane 0 reads the x-1 halo column, lane 31 the x+1 one (other lanes: any)
  const int hside = lane == 31 ? SIDE_XP : SIDE_XM;
  // FP64 resident and bands: when any strip of the launch has dead columns
  // every strip sweeps with the dead-column code, so that an SM's warps run
  // one instantiation of the long integer-path loop (the two side by side
  // measured 20% slower, and in these schedules every strip of a grid waits
  // for the slowest; tiles measured no gain)
  const bool any_dead = (sizeof(T) == 8 && kp.dead_all) || __any_sync(0xffffffffu, dead != 0);
  for (int t = 0; t < k; ++t) {
    if (act) {
      const int par = t & 1;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (remote[s]) wait_flag(kp.gflags + st.link[s], true, base + t, kp);
      if constexpr (kLocalFlags) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (local[s]) wait_flag(sflags + st.link[s] % NW, false, base + t, kp);
      }
      // halos of state t: rows into registers; remote columns staged into shared memory
      T hym[V], hyp[V];
      vload(inbox[SIDE_YM] + par * SW + lane * V, remote[SIDE_YM], hym);
      vload(inbox[SIDE_YP] + par * SW + lane * V, remote[SIDE_YP], hyp);
#pragma unroll
      for (int s = SIDE_XM; s <= SIDE_XP; ++s) {
        if (!remote[s]) continue;
        T *sb = mbox + L::side_off(s, rp) + par * rp;
        const T *gb = inbox[s] + par * rp;
        for (int r = lane; r < rows; r += 32) stm(&sb[r], ld_cg_chk(gb + r));
      }
      __syncwarp();
      const T *hcol = mbox + L::side_off(hside, rp) + par * rp;
      if constexpr (ADJ) {
        if (rg.ring) ring_accumulate(rg, data, drow, rows, lane);
      }
      if (any_dead)
        sweep_rows<T, ADJ, true>(drow, hcol, rows, lane, a, u, kp.int_path != 0, xl, st.y0, hym, hyp, dead, rg);
      else
        sweep_rows<T, ADJ, false>(drow, hcol, rows, lane, a, u, kp.int_path != 0, xl, st.y0, hym, hyp, dead, rg);
      __syncwarp();
      if (!ADJ && kp.states)  // a state-keeping run: this step's valid cells into their state
        strip_store_plain<T>(st, gd, drow, lane, reinterpret_cast<T *>(kp.states) + (size_t)(step0 + t) * kp.state_elems);
      publish_edges(par ^ 1);
      publish_local(base + t + 1);
      publish_remote(base + t + 1);
    }
    if constexpr (!kLocalFlags) __syncthreads();
  }
  if (!act) return;

  strip_store<T, ADJ>(st, gd, data, map_store, dstbuf, lane, rg);
}

// ---- two time steps per sweep (TILES, FP32 forward) -------------------------
//
// An exchange carries two steps.  A strip reads, in place from its neighbours'
// shared memory, the state-t cells two deep around it (rows -2, -1, R, R+1,
// columns -2, -1, SW, SW+1) and the four diagonal cells beside its corners,
// and evaluates step t+1 on the one-cell ring around itself exactly as the
// strip owning each of those cells does.  After a CTA barrier (every strip
// has read its neighbours) it sweeps its rows once, computing step t+1 of row
// r and step t+2 of row r-1 from two register windows, and stores step t+2 in
// place; a second barrier ends the exchange.  Per two steps: one shared-memory
// load and store per row, no mailbox copies, two CTA barriers.  Sides without
// a neighbour (ring, overlapped tile halo) keep the values read at the strip's
// load, as in the single-step exchange.

// One row (logical row y) of a sweep: new values from the old rows above
// (ra), at (rb) and below (rc); lane 0 takes x-1 from hl, lane 31 takes x+1
// from hr; dead columns keep their value.  The same evaluation as sweep_row()
// (FP64: the integer path on the cells exact_cell() selects).
template <typename T, bool DEAD>
__device__ __forceinline__ void row_update(const T (&ra)[VecOf<T>::V], const T (&rb)[VecOf<T>::V],
                                           const T (&rc)[VecOf<T>::V], T hl, T hr, int lane, const Links<T> &a,
                                           const ExactW &u, bool ipath, int xl, int y, uint32_t dead,
                                           T (&o)[VecOf<T>::V]) {
  constexpr int V = VecOf<T>::V;
  T left = __shfl_up_sync(0xffffffffu, rb[V - 1], 1);
  T right = __shfl_down_sync(0xffffffffu, rb[0], 1);
  if (lane == 0) left = hl;
  if (lane == 31) right = hr;
#pragma unroll
  for (int e = 0; e < V; ++e) {
    if (kSkipDead<T> && DEAD && (dead & (1u << e))) {  // as in sweep_row
      o[e] = rb[e];
      continue;
    }
    const T xm = e == 0 ? left : rb[e - 1], xp = e == V - 1 ? right : rb[e + 1];
    if constexpr (std::is_same<T, double>::value)
      o[e] = stencil_cell(a, u, exact_cell(xl + e, y, ipath), xm, xp, ra[e], rb[e], rc[e]);
    else
      o[e] = stencil(a, xm, xp, ra[e], rb[e], rc[e]);
  }
  if constexpr (!kSkipDead<T> && DEAD) {
#pragma unroll
    for (int e = 0; e < V; ++e)
      if (dead & (1u << e)) o[e] = rb[e];
  }
}

// Two steps over a strip in one pass.  hct / hct1: this lane's halo column
// (x-1 for lane 0, x+1 for lane 31) at steps t and t+1, one entry per row;
// m1 / m1n: row -1 at t / t+1; p0 / p0n: row R at t / t+1.
template <typename T, bool DEAD>
__device__ __forceinline__ void sweep_pair(T *drow, const T *hct, const T *hct1, int rows, int lane,
                                           const Links<T> &a, const ExactW &u, bool ip, int xl, int y0,
                                           const T (&m1)[VecOf<T>::V],
                                           const T (&m1n)[VecOf<T>::V], const T (&p0)[VecOf<T>::V],
                                           const T (&p0n)[VecOf<T>::V], uint32_t dead) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  T a0[V], b0[V], c0[V], a1[V], b1[V], n1[V], o[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    a0[e] = m1[e];
    a1[e] = m1n[e];
  }
  vload(drow, false, b0);
  if (rows > 1) {
    vload(drow + SW, false, c0);
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) c0[e] = p0[e];
  }
  row_update<T, DEAD>(a0, b0, c0, ldm(&hct[0]), ldm(&hct[0]), lane, a, u, ip, xl, y0, dead, b1);  // step t+1 of row 0
#pragma unroll
  for (int e = 0; e < V; ++e) {
    a0[e] = b0[e];
    b0[e] = c0[e];
  }
  // both windows advance by one row per iteration: unrolling by their period
  // (3) lets the compiler rename the registers instead of moving them (FP32;
  // the FP64 rows, with the integer path, do not fit three to a body); the
  // last row is peeled so that the loop loads the next row unconditionally
  constexpr int kUnroll = sizeof(T) == 4 ? 3 : 1;
#pragma unroll kUnroll
  for (int r = 1; r < rows - 1; ++r) {
    vload(drow + (r + 1) * SW, false, c0);
    row_update<T, DEAD>(a0, b0, c0, ldm(&hct[r]), ldm(&hct[r]), lane, a, u, ip, xl, y0 + r, dead, n1);  // step t+1 of row r
    row_update<T, DEAD>(a1, b1, n1, ldm(&hct1[r - 1]), ldm(&hct1[r - 1]), lane, a, u, ip, xl, y0 + r - 1, dead, o);  // t+2, row r-1
    vstore(drow + (r - 1) * SW, o);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      a1[e] = b1[e];
      b1[e] = n1[e];
      a0[e] = b0[e];
      b0[e] = c0[e];
    }
  }
  if (rows > 1) {
    const int r = rows - 1;
    row_update<T, DEAD>(a0, b0, p0, ldm(&hct[r]), ldm(&hct[r]), lane, a, u, ip, xl, y0 + r, dead, n1);  // step t+1 of the last row
    row_update<T, DEAD>(a1, b1, n1, ldm(&hct1[r - 1]), ldm(&hct1[r - 1]), lane, a, u, ip, xl, y0 + r - 1, dead, o);  // t+2, row R-2
    vstore(drow + (r - 1) * SW, o);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      a1[e] = b1[e];
      b1[e] = n1[e];
    }
  }
  row_update<T, DEAD>(a1, b1, p0n, ldm(&hct1[rows - 1]), ldm(&hct1[rows - 1]), lane, a, u, ip, xl, y0 + rows - 1, dead, o);  // t+2, last row
  vstore(drow + (rows - 1) * SW, o);
}

// Advance one tile strip by k steps, two per exchange (an odd k ends with one
// single step).  Called by every warp of the CTA with the same k.
template <typename T>
__device__ void run_strip_pair(const Strip &st, const KParams &kp, char *smem, int warp, int src, int dst, int k,
                               uint32_t &mbar_phase) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  const int lane = threadIdx.x & 31;
  const int region = pair_region_elems((int)sizeof(T), kp.rmax);
  T *wbase = reinterpret_cast<T *>(smem + kHeaderBytes);
  T *data = wbase + (size_t)warp * region;
  T *hc = data + (size_t)kp.rmax * SW;  // [4][32]: columns -1 and SW at step t, then at step t+1
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  const bool act = st.active;
  const GridDev &gd = kp.grids[act ? st.g : 0];
  const int nx = gd.nx, ny = gd.ny, rows = st.rows;
  const long pitch = gd.pitch;
  const int off = gd.off;
  const T *srcbuf = reinterpret_cast<const T *>(gd.buf[src]);
  T *dstbuf = reinterpret_cast<T *>(gd.buf[dst]);
  const CUtensorMap *map_load = kp.maps + (size_t)st.g * 6 + src;
  const CUtensorMap *map_store = kp.maps + (size_t)st.g * 6 + 3 + dst;
  const Links<T> a{(T)gd.w[0], (T)gd.w[1], (T)gd.w[2], (T)gd.w[3], (T)gd.w[4]};
  ExactW u{};
  if constexpr (std::is_same<T, double>::value) u = exact_weights(a);
  const bool ip = kp.int_path != 0;
  // a halo-column cell (logical x, y), evaluated as its owner evaluates it
  auto cell = [&](int x, int y, T xm, T xp, T ym, T c, T yp) -> T {
    if constexpr (std::is_same<T, double>::value)
      return stencil_cell(a, u, exact_cell(x, y, ip), xm, xp, ym, c, yp);
    else
      return stencil(a, xm, xp, ym, c, yp);
  };

  // neighbours (warps of this CTA: a tile has no other links) and the
  // diagonal strips, which exist whenever both adjacent neighbours do
  const int WX = st.tw;
  auto nbw = [&](int s) { return act && st.link[s] >= 0 ? st.link[s] % kWarps : -1; };
  const int wT = nbw(SIDE_YM), wB = nbw(SIDE_YP), wL = nbw(SIDE_XM), wR = nbw(SIDE_XP);
  const int wTL = wT >= 0 && wL >= 0 ? warp - WX - 1 : -1;
  const int wTR = wT >= 0 && wR >= 0 ? warp - WX + 1 : -1;
  const int wBL = wB >= 0 && wL >= 0 ? warp + WX - 1 : -1;
  const int wBR = wB >= 0 && wR >= 0 ? warp + WX + 1 : -1;
  const int trows = kp.tile_rows;  // the strip above is a full strip
  const int rowsB = wB >= 0 ? min(trows, ny + 1 - (st.y0 + rows)) : 0;
  auto nbdata = [&](int w) { return wbase + (size_t)w * region; };

  const int xl = st.x0 + lane * V;
  T *drow = data + lane * V;
  uint32_t dead = 0;
#pragma unroll
  for (int e = 0; e < V; ++e)
    if (act && xl + e > nx) dead |= 1u << e;

  // state-t cells around the strip (constant on sides without a neighbour)
  T hm2[V], hm1[V], hp0[V], hp1[V];                   // rows -2, -1, R, R+1
  T xm2 = T(0), xm1 = T(0), xp0 = T(0), xp1 = T(0);  // columns -2, -1, SW, SW+1 of row `lane`
  T ctl = T(0), ctr = T(0), cbl = T(0), cbr = T(0);  // the diagonal cells
  auto gval = [&](int y, int x) -> T {
    return (x >= 0 && x <= nx + 1 && y >= 0 && y <= ny + 1) ? ldm(&srcbuf[(long)y * pitch + off + x]) : T(0);
  };
  if (act) {
    fence_proxy_async_all();  // earlier generic writes before the async-proxy load
    __syncwarp();
    if (lane == 0) {
      bulk_wait_read_all();  // previous strip's stores have read shared memory
      const uint32_t bytes = (uint32_t)(SW * kp.rmax * sizeof(T));
      const bool ok = !kChecked || access_ok(data, bytes);  // a refused load still completes the phase
      mbar_expect_tx(&bars[warp], ok ? bytes : 0u);
      if (ok) tma_load_2d(data, map_load, off + st.x0, st.y0, &bars[warp]);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int x = xl + e;
      hm2[e] = wT < 0 ? gval(st.y0 - 2, x) : T(0);
      hm1[e] = wT < 0 ? gval(st.y0 - 1, x) : T(0);
      hp0[e] = wB < 0 ? gval(st.y0 + rows, x) : T(0);
      hp1[e] = (wB < 0 || rowsB < 2) ? gval(st.y0 + rows + 1, x) : T(0);
    }
    if (lane < rows) {
      const int y = st.y0 + lane;
      if (wL < 0) {
        xm2 = gval(y, st.x0 - 2);
        xm1 = gval(y, st.x0 - 1);
      }
      if (wR < 0) {
        xp0 = gval(y, st.x0 + SW);
        xp1 = gval(y, st.x0 + SW + 1);
      }
    }
    if (wTL < 0) ctl = gval(st.y0 - 1, st.x0 - 1);
    if (wTR < 0) ctr = gval(st.y0 - 1, st.x0 + SW);
    if (wBL < 0) cbl = gval(st.y0 + rows, st.x0 - 1);
    if (wBR < 0) cbr = gval(st.y0 + rows, st.x0 + SW);
    wait_mbar(&bars[warp], mbar_phase, kp);
    mbar_phase ^= 1u;
  }
  __syncthreads();

  const T *hct = hc + (lane == 31 ? 32 : 0);  // this lane's halo column at step t
  const T *hct1 = hct + 64;                   // and at step t+1
  const bool any_dead = __any_sync(0xffffffffu, dead != 0);
  for (int t = 0; t < k; t += 2) {
    const bool two = t + 1 < k;
    T m1n[V], p0n[V];
    if (act) {
      // the neighbours' state-t cells, read in place
      if (wT >= 0) {
        const T *d = nbdata(wT) + lane * V;
        vload(d + (trows - 2) * SW, false, hm2);
        vload(d + (trows - 1) * SW, false, hm1);
      }
      if (wB >= 0) {
        const T *d = nbdata(wB) + lane * V;
        vload(d, false, hp0);
        if (rowsB > 1) vload(d + SW, false, hp1);
      }
      if (lane < rows) {
        if (wL >= 0) {
          const T *d = nbdata(wL) + lane * SW;
          xm2 = ldm(&d[SW - 2]);
          xm1 = ldm(&d[SW - 1]);
        }
        if (wR >= 0) {
          const T *d = nbdata(wR) + lane * SW;
          xp0 = ldm(&d[0]);
          xp1 = ldm(&d[1]);
        }
      }
      if (wTL >= 0) ctl = ldm(&nbdata(wTL)[(trows - 1) * SW + SW - 1]);
      if (wTR >= 0) ctr = ldm(&nbdata(wTR)[(trows - 1) * SW]);
      if (wBL >= 0) cbl = ldm(&nbdata(wBL)[SW - 1]);
      if (wBR >= 0) cbr = ldm(&nbdata(wBR)[0]);
      if (two) {
        // step t+1 on the ring around the strip
        T own0 = T(0), ownl = T(0);
        if (lane < rows) {
          own0 = ldm(&data[lane * SW]);
          ownl = ldm(&data[lane * SW + SW - 1]);
        }
        T up = __shfl_up_sync(0xffffffffu, xm1, 1), dn = __shfl_down_sync(0xffffffffu, xm1, 1);
        if (lane == 0) up = ctl;
        if (lane == rows - 1) dn = cbl;
        const T l1 = wL >= 0 ? cell(st.x0 - 1, st.y0 + lane, xm2, own0, up, xm1, dn) : xm1;
        up = __shfl_up_sync(0xffffffffu, xp0, 1);
        dn = __shfl_down_sync(0xffffffffu, xp0, 1);
        if (lane == 0) up = ctr;
        if (lane == rows - 1) dn = cbr;
        const T r1 = wR >= 0 ? cell(st.x0 + SW, st.y0 + lane, ownl, xp1, up, xp0, dn) : xp0;
        if (lane < rows) {
          stm(&hc[64 + lane], l1);
          stm(&hc[96 + lane], r1);
        }
        T own[V];
        if (wT >= 0) {
          vload(drow, false, own);
          row_update<T, true>(hm2, hm1, own, ctl, ctr, lane, a, u, ip, xl, st.y0 - 1, dead, m1n);
        } else {
#pragma unroll
          for (int e = 0; e < V; ++e) m1n[e] = hm1[e];
        }
        if (wB >= 0) {
          vload(drow + (rows - 1) * SW, false, own);
          row_update<T, true>(own, hp0, hp1, cbl, cbr, lane, a, u, ip, xl, st.y0 + rows, dead, p0n);
        } else {
#pragma unroll
          for (int e = 0; e < V; ++e) p0n[e] = hp0[e];
        }
      }
      if (lane < rows) {
        stm(&hc[lane], xm1);
        stm(&hc[32 + lane], xp0);
      }
    }
    __syncthreads();  // every strip has read its neighbours' state-t cells
    if (act) {
      if (two) {
        if (any_dead)
          sweep_pair<T, true>(drow, hct, hct1, rows, lane, a, u, ip, xl, st.y0, hm1, m1n, hp0, p0n, dead);
        else
          sweep_pair<T, false>(drow, hct, hct1, rows, lane, a, u, ip, xl, st.y0, hm1, m1n, hp0, p0n, dead);
      } else {
        RingAcc<T> rg{};
        if (any_dead)
          sweep_rows<T, false, true>(drow, hct, rows, lane, a, u, ip, xl, st.y0, hm1, hp0, dead, rg);
        else
          sweep_rows<T, false, false>(drow, hct, rows, lane, a, u, ip, xl, st.y0, hm1, hp0, dead, rg);
      }
    }
    __syncthreads();  // every strip has written its new state
  }
  if (!act) return;
  const RingAcc<T> rg{};
  strip_store<T, false>(st, gd, data, map_store, dstbuf, lane, rg);
}

// ---- skewed serial tiles (SKEWED) -------------------------------------------
//
// Sections 3.1-3.3 and Figure 1 advance tiles one after another.  With a
// k-deep overlapped halo each tile recomputes its neighbours' edge cells; in
// skewed coordinates a tile takes them from its predecessor instead.  Skewed
// row q at time level t holds physical row y = q - t.  An update to level
// t+1 then reads, at level t, the skewed rows q-2 (the y-1 link), q-1 (the
// centre and its x-1 and x+1 links) and q (the y+1 link): the row itself and
// rows above it, never rows below.  So a column band is advanced k levels
// tile after tile from the top: a tile needs, at every level, the last two
// rows of the tile above it, and no halo below.  A CTA owns a contiguous run
// of the skewed rows of one or more column bands (a "piece" per band) and
// processes its tiles in order, handing the last two rows of each level to
// the next tile through a per-CTA buffer in global memory (double-buffered by
// tile parity).  A piece that starts inside a band starts 2(k-1) rows early:
// its top halo holds the level-0 rows at every level, which spoils 2(j-1)
// rows by level j.  Columns keep the overlapped halo of the TILES schedule.
// Cells whose physical row lies outside the interior (the ring rows, rows
// beyond the array) take the identity update, i.e. the value of their centre
// operand; the ring columns are read at the shifted row.  Every cell is
// evaluated with the same operands in the same order as in the one-step
// kernel, so results are bit-identical.  Inside a tile the neighbours' cells
// are read in place between two CTA barriers per step.

// A warp's region: its strip (R rows) and two 32-entry halo columns.
__host__ __device__ inline int skew_region_elems(int elem, int rmax) {
  const int SW = 32 * (16 / elem);
  const int per128 = 128 / elem;
  return (rmax * SW + 64 + per128 - 1) / per128 * per128;
}
__host__ __device__ inline size_t skew_smem_bytes(int elem, int rmax) {
  return (size_t)kHeaderBytes + (size_t)kWarps * skew_region_elems(elem, rmax) * elem;
}

// One step over a strip in skewed coordinates, swept top-down and updated in
// place: new row r from the old rows r-2 (the y-1 link), r-1 (the centre with
// its x-1 and x+1 links) and r (the y+1 link); ta, tb are rows -2 and -1.
// Rows [r_lo, r_hi) take the stencil, the others (physical row outside the
// interior) the identity.  yb: physical row of new row 0.
template <typename T, bool DEAD>
__device__ __forceinline__ void sweep_skew(T *drow, const T *hct, int rows, int r_lo, int r_hi, int lane,
                                           const Links<T> &a, const ExactW &u, bool ip, int xl, int yb,
                                           const T (&ta)[VecOf<T>::V], const T (&tb)[VecOf<T>::V],
                                           uint32_t dead) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  T ra[V], rb[V], rc[V], o[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    ra[e] = ta[e];
    rb[e] = tb[e];
  }
  int r = 0;
  for (; r < r_lo; ++r) {
    vload(drow + r * SW, false, rc);
    vstore(drow + r * SW, rb);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      ra[e] = rb[e];
      rb[e] = rc[e];
    }
  }
  // every row loads itself (no halo below): the body is the same for all
  // rows, unrolled by the window's period for FP32 as in sweep_rows
  constexpr int kUnroll = sizeof(T) == 4 ? 3 : 2;
#pragma unroll kUnroll
  for (; r < r_hi; ++r) {
    vload(drow + r * SW, false, rc);
    row_update<T, DEAD>(ra, rb, rc, ldm(&hct[r]), ldm(&hct[r]), lane, a, u, ip, xl, yb + r, dead, o);
    vstore(drow + r * SW, o);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      ra[e] = rb[e];
      rb[e] = rc[e];
    }
  }
  for (; r < rows; ++r) {
    vload(drow + r * SW, false, rc);
    vstore(drow + r * SW, rb);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      ra[e] = rb[e];
      rb[e] = rc[e];
    }
  }
}

// The same step for the 3x3 box: every row's x-1 / x+1 neighbours enter
// (shuffles; lane 0 and lane 31 take the halo column, hct[j] = strip row j-2).
template <typename T, bool DEAD>
__device__ __forceinline__ void sweep_skew_box(T *drow, const T *hct, int rows, int r_lo, int r_hi, int lane,
                                               const Box9<T> &b, const ExactWN<9> &u, bool ip, int xl, int yb,
                                               const T (&ta)[VecOf<T>::V], const T (&tb)[VecOf<T>::V],
                                               uint32_t dead) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  T ra[V], rb[V], rc[V], o[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    ra[e] = ta[e];
    rb[e] = tb[e];
  }
  auto sides = [&](const T (&row)[V], T h, T &l, T &r) {
    l = __shfl_up_sync(0xffffffffu, row[V - 1], 1);
    r = __shfl_down_sync(0xffffffffu, row[0], 1);
    if (lane == 0) l = h;
    if (lane == 31) r = h;
  };
  T al, ar, bl, br, cl, cr;
  sides(ra, ldm(&hct[0]), al, ar);
  sides(rb, ldm(&hct[1]), bl, br);
  auto shift = [&]() {
#pragma unroll
    for (int e = 0; e < V; ++e) {
      ra[e] = rb[e];
      rb[e] = rc[e];
    }
    al = bl;
    ar = br;
    bl = cl;
    br = cr;
  };
  int r = 0;
  for (; r < r_lo; ++r) {
    vload(drow + r * SW, false, rc);
    sides(rc, ldm(&hct[r + 2]), cl, cr);
    vstore(drow + r * SW, rb);
    shift();
  }
  for (; r < r_hi; ++r) {
    vload(drow + r * SW, false, rc);
    sides(rc, ldm(&hct[r + 2]), cl, cr);
    const int y = yb + r;
#pragma unroll
    for (int e = 0; e < V; ++e) {
      if (kSkipDead<T> && DEAD && (dead & (1u << e))) {  // as in sweep_row
        o[e] = rb[e];
        continue;
      }
      const T m0 = e == 0 ? al : ra[e - 1], m2 = e == V - 1 ? ar : ra[e + 1];
      const T c0 = e == 0 ? bl : rb[e - 1], c2 = e == V - 1 ? br : rb[e + 1];
      const T p0 = e == 0 ? cl : rc[e - 1], p2 = e == V - 1 ? cr : rc[e + 1];
      o[e] = stencil_box_cell(b, u, exact_cell(xl + e, y, ip), m0, ra[e], m2, c0, rb[e], c2, p0, rc[e], p2);
      if (!kSkipDead<T> && DEAD && (dead & (1u << e))) o[e] = rb[e];
    }
    vstore(drow + r * SW, o);
    shift();
  }
  for (; r < rows; ++r) {
    vload(drow + r * SW, false, rc);
    vstore(drow + r * SW, rb);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      ra[e] = rb[e];
      rb[e] = rc[e];
    }
  }
}

// Advance this warp's strip of one skewed tile (job) by k levels: load level
// 0, k steps, store level k.  Called by every warp of the CTA with the same k.
template <typename T, int NP>
__device__ void run_strip_skew(const KParams &kp, const int *job, char *smem, int warp, int src, int dst, int k,
                               int par, uint32_t &mbar_phase, const Prefetch &pf) {
  constexpr int V = VecOf<T>::V;
  constexpr int SW = 32 * V;
  const int lane = threadIdx.x & 31;
  const int R = kp.rmax;
  const int region = skew_region_elems((int)sizeof(T), R);
  T *wbase = reinterpret_cast<T *>(smem + kHeaderBytes);
  T *data = wbase + (size_t)warp * region;
  // [2][32]: halo column x-1 (then x+SW), entry j = strip row j - H0 (the
  // five-point cell reads the centre row's neighbours, rows -1 .. R-2; the
  // box cell all three rows', rows -2 .. R-1)
  T *hc = data + (size_t)R * SW;
  constexpr int H0 = NP == 9 ? 2 : 1;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  const int g = job[0], tx0 = job[1], vx0 = job[2], vx1 = job[3], q0 = job[4], nq = job[5], v0 = job[6],
            v1 = job[7];
  const bool first = job[8] != 0;
  const int wxa = job[9];
  const int WX = kp.skew_wx;
  const int wx = warp % WX, wy = warp / WX;
  const GridDev &gd = kp.grids[g];
  const int nx = gd.nx, ny = gd.ny;
  const long pitch = gd.pitch;
  const int off = gd.off;
  const int x0 = tx0 + wx * SW, y0 = q0 + wy * R;
  const int rows = min(R, q0 + nq - y0);
  const bool act = wx < wxa && rows > 0;
  const T *srcbuf = reinterpret_cast<const T *>(gd.buf[src]);
  T *dstbuf = reinterpret_cast<T *>(gd.buf[dst]);
  const CUtensorMap *map_load = kp.maps + (size_t)g * 6 + src;
  const CUtensorMap *map_store = kp.maps + (size_t)g * 6 + 3 + dst;
  const Links<T> a{(T)gd.w[0], (T)gd.w[1], (T)gd.w[2], (T)gd.w[3], (T)gd.w[4]};
  ExactW u{};
  Box9<T> b9{};
  ExactWN<9> u9{};
  if constexpr (NP == 9) {
    b9 = box_chain<T>(gd.w);
    if constexpr (std::is_same<T, double>::value) u9 = box_exact_weights(b9);
  } else {
    if constexpr (std::is_same<T, double>::value) u = exact_weights(a);
  }
  const bool ip = kp.int_path != 0;
  // neighbours in the tile (the strip above is full whenever this one has rows)
  const int wT = wy > 0 ? warp - WX : -1;
  const int wL = wx > 0 ? warp - 1 : -1;
  const int wR = wx + 1 < wxa ? warp + 1 : -1;
  const int wTL = wT >= 0 && wL >= 0 ? warp - WX - 1 : -1;
  const int wTR = wT >= 0 && wR >= 0 ? warp - WX + 1 : -1;
  auto nbdata = [&](int w) { return wbase + (size_t)w * region; };
  // the tile's last two rows at every level, for the next tile of the piece
  T *sbuf = reinterpret_cast<T *>(kp.skewbuf) + (size_t)blockIdx.x * 2 * kp.skew_levels * 2 * kp.skew_tw;
  auto sb = [&](int p, int lev, int row) { return sbuf + (((size_t)p * kp.skew_levels + lev) * 2 + row) * kp.skew_tw; };
  const bool bottom = act && rows >= 2 && y0 + rows == q0 + nq;
  auto gval = [&](int y, int x) -> T {
    return (x >= 0 && x <= nx + 1 && y >= 0 && y <= ny + 1) ? ldm(&srcbuf[(long)y * pitch + off + x]) : T(0);
  };

  const int xl = x0 + lane * V;
  T *drow = data + lane * V;
  uint32_t dead = 0;
#pragma unroll
  for (int e = 0; e < V; ++e)
    if (act && xl + e > nx) dead |= 1u << e;

  // level-0 halo above a tile-top strip and the two level-0 corner cells
  T t2c[V], t1c[V];
  T cl0 = T(0), cr0 = T(0);
  if (act) {
    fence_proxy_async_all();  // earlier generic writes before the async-proxy load
    __syncwarp();
    if (lane == 0) {
      bulk_wait_read_all();  // previous tile's stores have read shared memory
      const uint32_t bytes = (uint32_t)(SW * R * sizeof(T));
      const bool ok = !kChecked || access_ok(data, bytes);  // a refused load still completes the phase
      mbar_expect_tx(&bars[warp], ok ? bytes : 0u);
      if (ok) tma_load_2d(data, map_load, off + x0, y0, &bars[warp]);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      t2c[e] = wT < 0 ? gval(y0 - 2, xl + e) : T(0);
      t1c[e] = wT < 0 ? gval(y0 - 1, xl + e) : T(0);
    }
    if (lane < H0) {  // the corner cells of halo rows -H0 .. -1, one per lane
      cl0 = gval(y0 - H0 + lane, x0 - 1);
      cr0 = gval(y0 - H0 + lane, x0 + SW);
    }
    wait_mbar(&bars[warp], mbar_phase, kp);
    mbar_phase ^= 1u;
    if (pf.map && lane == 0) tma_prefetch_2d(pf.map, pf.x, pf.y);
  }
  __syncthreads();  // every strip holds level 0

  const T *hct = hc + (lane == 31 ? 32 : 0);
  const bool any_dead = __any_sync(0xffffffffu, dead != 0);
  // values a tile-top or tile-edge strip takes from global memory, loaded one
  // level ahead (during the sweep before the step that reads them): the two
  // halo rows above (the level-0 rows for the first tile of a piece, else the
  // previous tile's rows), the two corner cells (lane 0) and the ring columns
  T pa[V], pb[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    pa[e] = t2c[e];
    pb[e] = t1c[e];
  }
  T pcl = cl0, pcr = cr0;
  T phl = x0 == 1 ? gval(y0 + lane - H0, 0) : T(0);
  T phr = x0 + SW == nx + 1 ? gval(y0 + lane - H0, nx + 1) : T(0);
  for (int L = 1; L <= k; ++L) {
    T ta[V], tb[V];  // rows -2 and -1 at level L-1
    if (act) {
      if (wT >= 0) {
        const T *d = nbdata(wT) + lane * V;
        vload(d + (R - 2) * SW, false, ta);
        vload(d + (R - 1) * SW, false, tb);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          ta[e] = pa[e];
          tb[e] = pb[e];
        }
      }
      if (lane < rows + 2 * (H0 - 1)) {
        // halo columns at strip row lane - H0 (level L-1; the ring columns
        // at the physical row y0 + lane - H0 - (L-1), loaded ahead)
        const int row = lane - H0;
        T hl, hr;
        if (wL >= 0)
          hl = row >= 0 ? ldm(&nbdata(wL)[row * SW + SW - 1]) : wTL >= 0 ? ldm(&nbdata(wTL)[(R + row) * SW + SW - 1]) : pcl;
        else
          hl = phl;  // the ring column, or zero at a band edge (overlapped halo)
        if (wR >= 0)
          hr = row >= 0 ? ldm(&nbdata(wR)[row * SW]) : wTR >= 0 ? ldm(&nbdata(wTR)[(R + row) * SW]) : pcr;
        else
          hr = phr;
        stm(&hc[lane], hl);
        stm(&hc[32 + lane], hr);
      }
    }
    __syncthreads();  // every strip has read its neighbours' level-(L-1) cells
    if (act) {
      if (L < k) {
        // the next level's values from global memory, in flight during the sweep
        if (wT < 0 && !first) {
          vload(sb(par ^ 1, L, 0) + (x0 - tx0) + lane * V, false, pa);
          vload(sb(par ^ 1, L, 1) + (x0 - tx0) + lane * V, false, pb);
          if (lane < H0) {
            if (wL >= 0) pcl = ldm(&sb(par ^ 1, L, 2 - H0 + lane)[x0 - 1 - tx0]);
            if (wR >= 0) pcr = ldm(&sb(par ^ 1, L, 2 - H0 + lane)[x0 + SW - tx0]);
          }
        }
        if (x0 == 1) phl = gval(y0 + lane - L - H0, 0);
        if (x0 + SW == nx + 1) phr = gval(y0 + lane - L - H0, nx + 1);
      }
      // rows whose physical row y0 + r - L is interior take the stencil, the rest the identity
      const int r_lo = min(max(L + 1 - y0, 0), rows), r_hi = max(min(ny + L + 1 - y0, rows), r_lo);
      if constexpr (NP == 9) {
        if (any_dead)
          sweep_skew_box<T, true>(drow, hct, rows, r_lo, r_hi, lane, b9, u9, ip, xl, y0 - L, ta, tb, dead);
        else
          sweep_skew_box<T, false>(drow, hct, rows, r_lo, r_hi, lane, b9, u9, ip, xl, y0 - L, ta, tb, dead);
      } else {
        if (any_dead)
          sweep_skew<T, true>(drow, hct, rows, r_lo, r_hi, lane, a, u, ip, xl, y0 - L, ta, tb, dead);
        else
          sweep_skew<T, false>(drow, hct, rows, r_lo, r_hi, lane, a, u, ip, xl, y0 - L, ta, tb, dead);
      }
      if (bottom && L < k) {
        __syncwarp();
        T v[V];
        vload(drow + (rows - 2) * SW, false, v);
        vstore(sb(par, L, 0) + (x0 - tx0) + lane * V, v);
        vload(drow + (rows - 1) * SW, false, v);
        vstore(sb(par, L, 1) + (x0 - tx0) + lane * V, v);
      }
    }
    if (L < k) __syncthreads();  // every strip holds level L
  }
  if (!act) return;
  // store level k: physical rows [v0, v1) are the skewed rows [v0+k, v1+k)
  Strip st{};
  st.g = g;
  st.x0 = x0;
  st.y0 = y0 - k;
  st.rows = rows;
  st.ring = 0;
  st.sy0 = max(v0 + k - y0, 0);
  st.sy1 = min(v1 + k - y0, rows);
  if (st.sy1 < st.sy0) st.sy1 = st.sy0;
  st.sx0 = max(vx0 - x0, 0);
  st.sx1 = min(min(vx1, nx + 1) - x0, SW);
  if (st.sx1 < st.sx0) st.sx1 = st.sx0;
  if (st.sx0 == 0 && x0 + st.sx1 >= min(vx1, nx + 1) && (vx1 > nx || st.sx1 == SW)) st.sx1 = SW;
  const RingAcc<T> rg{};
  strip_store<T, false>(st, gd, data, map_store, dstbuf, lane, rg);
}

// Strip of slot `slot` in a band wave: columns strip j, row strip i of m.
__device__ Strip band_strip(const KParams &kp, const int *wave, int slot, int SWc) {
  Strip st{};
  const GridDev &gd = kp.grids[0];
  const int nx = gd.nx, ny = gd.ny;
  const int by0 = wave[0], by1 = wave[1], vy0 = wave[2], vy1 = wave[3], m = wave[4];
  const int ncs = (nx + SWc - 1) / SWc;
  // strip (column j, row i) of slot: either consecutive slots run down a
  // column (bx = 0), or each CTA holds a block of bx columns x 16/bx rows, so
  // that most x neighbours share the CTA as well
  const int BX = kp.bx > 0 ? kp.bx : 1, BY = kWarps / BX, nbx = (ncs + BX - 1) / BX;
  int j, i;
  if (kp.bx == 0) {
    j = slot / m;
    i = slot % m;
    st.active = slot < ncs * m;
  } else {
    const int b = slot / kWarps, w = slot % kWarps;
    j = (b % nbx) * BX + w % BX;
    i = (b / nbx) * BY + w / BX;
    st.active = j < ncs && i < m;
  }
  if (!st.active) return st;
  auto slot_of = [&](int jj, int ii) {
    return kp.bx == 0 ? jj * m + ii : ((ii / BY) * nbx + jj / BX) * kWarps + (ii % BY) * BX + jj % BX;
  };
  // rows spread evenly: strip i gets one of the `extra` leftover rows when
  // floor((i+1)*extra/m) steps up, so every run of consecutive strips (a CTA)
  // carries the same work to within one row
  const int hb = by1 - by0, bsz = hb / m, extra = hb % m;
  const int before = (int)((long)i * extra / m), upto = (int)((long)(i + 1) * extra / m);
  st.g = 0;
  st.rows = bsz + (upto - before);
  st.y0 = by0 + i * bsz + before;
  st.x0 = 1 + j * SWc;
  st.active = st.rows > 0;
  const int ylast = st.y0 + st.rows - 1;
  st.ring = 0;
  if (st.y0 == 1) st.ring |= 1 << SIDE_YM;
  if (ylast == ny) st.ring |= 1 << SIDE_YP;
  if (st.x0 == 1) st.ring |= 1 << SIDE_XM;
  if (st.x0 <= nx && nx <= st.x0 + SWc - 1) st.ring |= 1 << SIDE_XP;
  st.link[SIDE_YM] = i > 0 ? slot_of(j, i - 1) : LINK_CONST;
  st.link[SIDE_YP] = i < m - 1 ? slot_of(j, i + 1) : LINK_CONST;
  st.link[SIDE_XM] = j > 0 ? slot_of(j - 1, i) : LINK_CONST;
  st.link[SIDE_XP] = j < ncs - 1 ? slot_of(j + 1, i) : LINK_CONST;
  st.sy0 = max(vy0 - st.y0, 0);
  st.sy1 = min(vy1 - st.y0, st.rows);
  if (st.sy1 < st.sy0) st.sy1 = st.sy0;
  st.sx0 = 0;
  st.sx1 = SWc;
  return st;
}

// Strip of warp w (counted from the tile's first warp) of a tile of WX x WY
// strips; rows per strip kp.tile_rows.
__device__ Strip tile_strip(const KParams &kp, const int *tile, int w, int cta_slot0, int SWc) {
  Strip st{};
  const int g = tile[0], tx0 = tile[1], ty0 = tile[2], vx0 = tile[3], vx1 = tile[4], vy0 = tile[5], vy1 = tile[6];
  const int WX = tile[8], WY = tile[9];
  cta_slot0 += tile[7];
  const GridDev &gd = kp.grids[g];
  const int nx = gd.nx, ny = gd.ny;
  const int wx = w % WX, wy = w / WX;
  st.tw = WX;
  st.g = g;
  st.x0 = tx0 + wx * SWc;
  st.y0 = ty0 + wy * kp.tile_rows;
  st.active = st.x0 <= nx && st.y0 <= ny;
  if (!st.active) return st;
  st.rows = min(kp.tile_rows, ny + 1 - st.y0);
  const int ylast = st.y0 + st.rows - 1;
  st.ring = 0;
  if (st.y0 == 1) st.ring |= 1 << SIDE_YM;
  if (ylast == ny) st.ring |= 1 << SIDE_YP;
  if (st.x0 == 1) st.ring |= 1 << SIDE_XM;
  if (st.x0 <= nx && nx <= st.x0 + SWc - 1) st.ring |= 1 << SIDE_XP;
  const bool up_ok = wy > 0;
  const bool dn_ok = wy < WY - 1 && ylast < ny;
  const bool lf_ok = wx > 0;
  const bool rt_ok = wx < WX - 1 && st.x0 + SWc <= nx;
  st.link[SIDE_YM] = up_ok ? cta_slot0 + w - WX : LINK_CONST;
  st.link[SIDE_YP] = dn_ok ? cta_slot0 + w + WX : LINK_CONST;
  st.link[SIDE_XM] = lf_ok ? cta_slot0 + w - 1 : LINK_CONST;
  st.link[SIDE_XP] = rt_ok ? cta_slot0 + w + 1 : LINK_CONST;
  st.sy0 = max(vy0 - st.y0, 0);
  st.sy1 = min(vy1 - st.y0, st.rows);
  if (st.sy1 < st.sy0) st.sy1 = st.sy0;
  st.sx0 = max(vx0 - st.x0, 0);
  st.sx1 = min(min(vx1, nx + 1) - st.x0, SWc);
  if (st.sx1 < st.sx0) st.sx1 = st.sx0;
  // a strip whose valid columns reach its end (or the last interior column)
  // is stored whole with TMA; the store map clips beyond column nx
  if (st.sx0 == 0 && st.x0 + st.sx1 >= min(vx1, nx + 1) && (vx1 > nx || st.sx1 == SWc)) st.sx1 = SWc;
  return st;
}

// This warp's strip in the tile group starting at job j (inactive if no tile
// of the group uses it); count = the group's number of tiles.
__device__ Strip group_strip(const KParams &kp, int j, int warp, int cta_slot0, int SWc, int &count) {
  const int *t0 = kp.jobs + (size_t)kTileInts * j;
  count = t0[10];
  for (int i = 0; i < count; ++i) {
    const int *t = t0 + (size_t)kTileInts * i;
    const int w = warp - t[7];
    if (w >= 0 && w < t[8] * t[9]) return tile_strip(kp, t, w, cta_slot0, SWc);
  }
  return Strip{};
}

// This slot's strip in a grouped-resident wave (the record holds it whole).
__device__ Strip slot_strip(const int *rec, int SWc) {
  Strip st{};
  st.active = rec[0] >= 0;
  if (!st.active) return st;
  st.g = rec[0];
  st.x0 = rec[1];
  st.y0 = rec[2];
  st.rows = rec[3];
  st.ring = rec[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) st.link[s] = rec[5 + s];
  st.sy0 = 0;
  st.sy1 = st.rows;
  st.sx0 = 0;
  st.sx1 = SWc;
  return st;
}

// Ring copy for every grid of a run in one launch: block (g, d) copies the
// ring of grid g's input to its buffer d (1 = workspace, 2 = output).
template <typename T>
__global__ void ring_copy_grids_kernel(const GridDev *grids, int copy_ws, int copy_out, unsigned long long mem_lo,
                                       unsigned long long mem_hi) {
#ifdef J2D_BOUNDS_CHECK
  if (threadIdx.x == 0) {
    s_mem_lo = mem_lo;
    s_mem_hi = mem_hi;
  }
  __syncthreads();
#else
  (void)mem_lo;
  (void)mem_hi;
#endif
  const GridDev &g = grids[blockIdx.x];
  const int d = blockIdx.y == 0 ? 2 : 1;
  if ((d == 2 && !copy_out) || (d == 1 && !copy_ws) || g.buf[d] == g.buf[0]) return;
  const T *in = reinterpret_cast<const T *>(g.buf[0]);
  T *out = reinterpret_cast<T *>(g.buf[d]);
  const int nx = g.nx, ny = g.ny, n_rows = 2 * (nx + 2), n = n_rows + 2 * ny;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int y, x;
    if (i < n_rows) {
      y = (i < nx + 2) ? 0 : ny + 1;
      x = i % (nx + 2);
    } else {
      const int j = i - n_rows;
      y = 1 + (j >> 1);
      x = (j & 1) ? nx + 1 : 0;
    }
    const long e = (long)y * g.pitch + g.off + x;
    stm(&out[e], ldm(&in[e]));
  }
}

template <typename T, bool ADJ, int MODE, int NP = 5>
__global__ void __launch_bounds__(kThreads, 1) dtb_kernel(const __grid_constant__ KParams kp) {
  constexpr int SWc = 32 * VecOf<T>::V;
  extern __shared__ __align__(1024) char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  int *sflags = reinterpret_cast<int *>(smem + 512);
  if (lane == 0) {
    mbar_init(&bars[warp], 1);
    sflags[warp] = -1;
  }
#ifdef J2D_BOUNDS_CHECK
  if (threadIdx.x == 0) {
    s_mem_lo = kp.mem_lo;
    s_mem_hi = kp.mem_hi;
  }
#endif
  fence_mbar_init();
  fence_proxy_async_smem();
  __syncthreads();
  uint32_t phase = 0;
  int epoch = 0;
  const int slot = blockIdx.x * kWarps + warp;
  const int kmax1 = max(kp.depth, kp.last_depth) + 1;
  int seq = 0;  // strips processed by this CTA (tiles) / waves (bands)
  for (int r = 0; r < kp.rounds; ++r) {
    const int dst = ((kp.rounds - 1 - r) & 1) == 0 ? 2 : 1;
    const int src = r == 0 ? kp.src0 : (((kp.rounds - r) & 1) == 0 ? 2 : 1);
    const int k = r == kp.rounds - 1 ? kp.last_depth : kp.depth;
    if constexpr (MODE == MODE_SKEW) {
      // this CTA's tiles in order; tile parity selects the halo-row buffer
      const int jend = kp.job_off[blockIdx.x + 1];
      int par = 0;
      for (int j = kp.job_off[blockIdx.x]; j < jend; ++j, par ^= 1) {
        const int *job = kp.jobs + (size_t)kSkewInts * j;
        // this warp's strip of the next tile goes into L2 while this one runs
        Prefetch pf;
        if (j + 1 < jend) {
          const int *nj = job + kSkewInts;
          const int wx = warp % kp.skew_wx, wy = warp / kp.skew_wx;
          if (wx < nj[9] && wy * kp.rmax < nj[5] && nj[4] + wy * kp.rmax <= kp.grids[nj[0]].ny + 1) {
            pf.map = kp.maps + (size_t)nj[0] * 6 + src;
            pf.x = kp.grids[nj[0]].off + nj[1] + wx * SWc;
            pf.y = nj[4] + wy * kp.rmax;
          }
        }
        run_strip_skew<T, NP>(kp, job, smem, warp, src, dst, k, par, phase, pf);
      }
      if (lane == 0) {
        bulk_wait_all();
        fence_proxy_async_global();
      }
      grid_barrier(kp, epoch);
    } else if (MODE == MODE_GROUPS) {
      // every wave is all k steps of its grids; the barrier after it also
      // keeps the next wave's edges out of mailboxes still being read
      const size_t nslots = (size_t)gridDim.x * kWarps;
      for (int wv = 0; wv < kp.njobs; ++wv, ++seq) {
        const Strip st = slot_strip(kp.jobs + ((size_t)wv * nslots + slot) * kSlotInts, SWc);
        run_strip<T, ADJ>(st, kp, smem, warp, slot, src, dst, k, seq * kmax1, phase);
        if (lane == 0) {
          bulk_wait_all();
          fence_proxy_async_global();
        }
        grid_barrier(kp, epoch);
      }
    } else if (MODE == MODE_BANDS) {
      for (int wv = 0; wv < kp.njobs; ++wv, ++seq) {
        const Strip st = band_strip(kp, kp.jobs + 5 * wv, slot, SWc);
        run_strip<T, ADJ>(st, kp, smem, warp, slot, src, dst, k, seq * kmax1, phase, Prefetch{}, r * kp.depth);
        if (lane == 0) {
          bulk_wait_all();
          fence_proxy_async_global();
        }
        grid_barrier(kp, epoch);
      }
    } else {
      int cnt = 1;
      for (int j = kp.job_off[blockIdx.x]; j < kp.job_off[blockIdx.x + 1]; j += cnt, ++seq) {
        const Strip st = group_strip(kp, j, warp, blockIdx.x * kWarps, SWc, cnt);
        if constexpr (MODE == MODE_TILES_PAIR) {
          run_strip_pair<T>(st, kp, smem, warp, src, dst, k, phase);
        } else {
          // this warp's strip of the CTA's next tile (same round, same source)
          // goes into L2 while this tile runs (+1% FP64 tiles; the two-step
          // FP32 kernel has no registers to spare for it: -2% there)
          Prefetch pf;
          if (j + cnt < kp.job_off[blockIdx.x + 1]) {
            int ncnt;
            const Strip nst = group_strip(kp, j + cnt, warp, blockIdx.x * kWarps, SWc, ncnt);
            if (nst.active) {
              pf.map = kp.maps + (size_t)nst.g * 6 + src;
              pf.x = kp.grids[nst.g].off + nst.x0;
              pf.y = nst.y0;
            }
          }
          run_strip<T, ADJ>(st, kp, smem, warp, slot, src, dst, k, seq * kmax1, phase, pf, r * kp.depth);
        }
        __syncthreads();
      }
      if (lane == 0) {
        bulk_wait_all();
        fence_proxy_async_global();
      }
      grid_barrier(kp, epoch);
    }
  }
  if (lane == 0) bulk_wait_all();
}

// ---- host side -------------------------------------------------------------

int dtb_rows_max(j2d_dtype dt, size_t smem_optin, int warps) {
  const int elem = dt == J2D_F64 ? 8 : 4;
  (void)warps;
  for (int r = 64; r >= 1; --r) {
    const int rp = (r + 3) / 4 * 4;
    if (dtb_smem_bytes(elem, r, rp) <= smem_optin) return r;
  }
  return 0;
}

int dtb_rows_max_pair(j2d_dtype dt, size_t smem_optin) {
  const int elem = dt == J2D_F64 ? 8 : 4;
  for (int r = 32; r >= 1; --r)
    if (pair_smem_bytes(elem, r) <= smem_optin) return r;
  return 0;
}

int dtb_rows_max_skew(j2d_dtype dt, size_t smem_optin) {
  const int elem = dt == J2D_F64 ? 8 : 4;
  for (int r = 32; r >= 2; --r)
    if (skew_smem_bytes(elem, r) <= smem_optin) return r;
  return 0;
}

static int vec_of(j2d_dtype dt) { return dt == J2D_F64 ? 2 : 4; }

// Resident fit: strips per column m and rows per strip for one grid on `ctas` CTAs.
static bool resident_fit(const GridDesc &g, int sw, int ctas, int rmax, int *m_out) {
  const int ncs = (g.nx + sw - 1) / sw;
  const long slots = (long)ctas * kWarps;
  if (ncs > slots) return false;
  int m = (int)std::min<long>(slots / ncs, g.ny);
  if ((g.ny + m - 1) / m > rmax) return false;
  *m_out = m;
  return true;
}

// Grouped resident (RESIDENT on a batch): every grid must fit the CTAs'
// warps by itself with strips of at most rmax rows.
static bool groups_fit(const std::vector<GridDesc> &grids, int sw, int ctas, int rmax) {
  const long slots = (long)ctas * kWarps;
  for (const GridDesc &g : grids)
    if ((long)((g.nx + sw - 1) / sw) * ((g.ny + rmax - 1) / rmax) > slots) return false;
  return true;
}

// The waves of a grouped-resident run, as kSlotInts records per slot and
// wave.  Grids are taken tallest strips first (then most strips) and each
// goes into the first wave with room for it (first fit, strips of rmax
// rows); then every wave takes the shortest strip height that still fits
// its grids, so an under-filled wave spreads over all warps (a wave lasts
// as long as its tallest strip: warps advance in step with their
// neighbours).  A grid's strips take consecutive slots, four strip
// columns at a time row by row, so that a CTA's 16 slots hold 4 x 4 strips
// and most links stay inside the CTA.  Returns the number of waves (0: a
// grid does not fit).
static int group_waves(const std::vector<GridDesc> &grids, int sw, int ctas, int rmax, std::vector<int> &jobs) {
  const int slots = ctas * kWarps;
  const int ng = (int)grids.size();
  if (!groups_fit(grids, sw, ctas, rmax)) return 0;
  std::vector<int> ncs(ng), order(ng);
  auto height = [&](int g, int h) {  // strip rows of grid g with strips of at most h rows
    const int m = (grids[g].ny + h - 1) / h;
    return (grids[g].ny + m - 1) / m;
  };
  auto strips = [&](int g, int h) { return (long)ncs[g] * ((grids[g].ny + h - 1) / h); };
  for (int g = 0; g < ng; ++g) {
    ncs[g] = (grids[g].nx + sw - 1) / sw;
    order[g] = g;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ha = height(a, rmax), hb = height(b, rmax);
    return ha != hb ? ha > hb : strips(a, rmax) > strips(b, rmax);
  });
  std::vector<std::vector<int>> waves;
  std::vector<long> used;
  for (int g : order) {
    const long n = strips(g, rmax);
    size_t w = 0;
    while (w < waves.size() && used[w] + n > slots) ++w;
    if (w == waves.size()) {
      waves.emplace_back();
      used.push_back(0);
    }
    waves[w].push_back(g);
    used[w] += n;
  }
  const int nw = (int)waves.size();
  jobs.assign((size_t)nw * slots * kSlotInts, 0);
  for (size_t i = 0; i < jobs.size(); i += kSlotInts) jobs[i] = -1;
  for (int w = 0; w < nw; ++w) {
    int h = 1;
    for (;; ++h) {
      long need = 0;
      for (int g : waves[w]) need += strips(g, h);
      if (need <= slots || h == rmax) break;
    }
    int s0 = 0;
    for (int g : waves[w]) {
      const GridDesc &gd = grids[g];
      const int nc = ncs[g], m = (gd.ny + h - 1) / h;
      // slot of strip column j, strip row i: groups of four columns, row-major inside a group
      auto slot_of = [&](int j, int i) {
        const int grp = j / 4, cw = std::min(4, nc - 4 * grp);
        return s0 + grp * 4 * m + i * cw + (j - 4 * grp);
      };
      const int bsz = gd.ny / m, extra = gd.ny % m;
      for (int j = 0; j < nc; ++j)
        for (int i = 0; i < m; ++i) {
          // rows spread as in the bands: strip i takes one of the leftover rows when floor(i*extra/m) steps up
          const int before = (int)((long)i * extra / m), upto = (int)((long)(i + 1) * extra / m);
          const int rows = bsz + (upto - before), y0 = 1 + i * bsz + before, x0 = 1 + j * sw;
          int ring = 0;
          if (y0 == 1) ring |= 1 << SIDE_YM;
          if (y0 + rows - 1 == gd.ny) ring |= 1 << SIDE_YP;
          if (x0 == 1) ring |= 1 << SIDE_XM;
          if (gd.nx <= x0 + sw - 1) ring |= 1 << SIDE_XP;
          int *rec = &jobs[((size_t)w * slots + slot_of(j, i)) * kSlotInts];
          rec[0] = g;
          rec[1] = x0;
          rec[2] = y0;
          rec[3] = rows;
          rec[4] = ring;
          rec[5 + SIDE_YM] = i > 0 ? slot_of(j, i - 1) : LINK_CONST;
          rec[5 + SIDE_YP] = i < m - 1 ? slot_of(j, i + 1) : LINK_CONST;
          rec[5 + SIDE_XM] = j > 0 ? slot_of(j - 1, i) : LINK_CONST;
          rec[5 + SIDE_XP] = j < nc - 1 ? slot_of(j + 1, i) : LINK_CONST;
        }
      s0 += nc * m;
    }
  }
  return nw;
}

// Strips per column for one grid of ncs strip columns on `ctas` CTAs when
// each CTA holds a block of bx columns x 16/bx rows of strips (bx = 0:
// consecutive slots run down the columns); 0 if the grid is too wide.
static int strips_per_column(int ncs, int ny, int ctas, int bx) {
  if (bx == 0) {
    const long slots = (long)ctas * kWarps;
    return ncs > slots ? 0 : (int)std::min<long>(slots / ncs, ny);
  }
  const int nbx = (ncs + bx - 1) / bx;
  return nbx > ctas ? 0 : std::min((kWarps / bx) * (ctas / nbx), ny);
}

// The strip mapping of RESIDENT / BANDS: the most strips per column (the
// least work per warp); among equals, the CTA block with the fewest strip
// edges leaving the CTA (4x4, then 8x2, then 2x8, then columns).
static int choose_bx(int ncs, int ny, int ctas, int *m_out) {
  int best_bx = 0, best_m = strips_per_column(ncs, ny, ctas, 0);
  for (int bx : {2, 8, 4}) {
    const int m = strips_per_column(ncs, ny, ctas, bx);
    if (m > 0 && m >= best_m) {
      best_bx = bx;
      best_m = m;
    }
  }
  *m_out = best_m;
  return best_bx;
}

DtbConfig dtb_choose(j2d_dtype dt, const std::vector<GridDesc> &grids, int sms, size_t smem_optin,
                     const DtbRequest &rq) {
  DtbConfig c;
  c.ctas = rq.ctas > 0 ? std::min(rq.ctas, sms) : sms;
  c.rows = dtb_rows_max(dt, smem_optin, kWarps);
  const int sw = 32 * vec_of(dt);
  int algo = rq.algo;
  const bool single = grids.size() == 1;
  int m = 0;
  const bool fits = single ? resident_fit(grids[0], sw, c.ctas, c.rows, &m)
                           : !rq.adjoint && groups_fit(grids, sw, c.ctas, c.rows);
  if (algo == J2D_ALGO_AUTO) {
    if (rq.steps < 4) algo = J2D_ALGO_ONESTEP;
    else if (fits && (single || dt == J2D_F64)) algo = J2D_ALGO_RESIDENT;  // FP64 batches: grouped resident
    // grids too large for the chip: the stream schedule for FP32 (16384^2:
    // 4254 GCells/s against 1950 for the best shared-memory schedule; the box
    // 2578 against 1418) and for large FP64 grids (16384^2: 194 against 162 for
    // the tiles; 8192^2: 170; at 4096^2 the tiles are faster, 143 against 130)
    else if (single && !rq.adjoint && (dt == J2D_F32 || (long)grids[0].nx * grids[0].ny >= (8192L << 13)))
      algo = J2D_ALGO_STREAM;
    else algo = J2D_ALGO_TILES;
  }
  if (algo == J2D_ALGO_RESIDENT && !fits) algo = single ? J2D_ALGO_BANDS : J2D_ALGO_TILES;
  if (algo == J2D_ALGO_BANDS && !single) algo = J2D_ALGO_TILES;
  if (algo == J2D_ALGO_SKEWED && rq.adjoint) algo = J2D_ALGO_TILES;  // the skewed order is forward only
  if (algo == J2D_ALGO_STREAM && (rq.adjoint || !single)) algo = J2D_ALGO_TILES;  // forward, one grid
  // the 3x3 box runs the one-step kernel, the skewed tiles or the stream schedule
  if (grids[0].shape == 9 && algo != J2D_ALGO_ONESTEP && algo != J2D_ALGO_STREAM) algo = J2D_ALGO_SKEWED;
  c.algo = algo;
  c.depth = rq.depth > 0 ? rq.depth : (dt == J2D_F64 ? 4 : 8);
  c.tile_wx = rq.tile_wx > 0 ? rq.tile_wx : (dt == J2D_F64 ? 4 : 2);
  if (algo == J2D_ALGO_RESIDENT) c.depth = (int)std::max<long>(rq.steps, 1);
  // two steps per sweep: FP32 only (FP64 tiles measured 11% slower with it:
  // the integer path of four cells in flight spills at 128 registers)
  if (algo == J2D_ALGO_TILES && dt == J2D_F32 && !rq.adjoint && rq.sweep_steps == 2) {
    c.sweep = 2;
    c.rows = dtb_rows_max_pair(dt, smem_optin);
  }
  if (algo == J2D_ALGO_STREAM && rq.depth <= 0) c.depth = dt == J2D_F64 ? 2 : 8;
  if (algo == J2D_ALGO_SKEWED) {
    c.rows = dtb_rows_max_skew(dt, smem_optin);
    if (rq.depth <= 0) c.depth = dt == J2D_F64 ? 8 : 16;
    if (rq.tile_wx <= 0) c.tile_wx = 4;
  }
  return c;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool encode_map(CUtensorMap *m, j2d_dtype dt, void *base, long pitch, long width, long height, int boxw,
                       int boxh) {
  auto enc = get_encoder();
  if (!enc) return false;
  const size_t elem = dt == J2D_F64 ? 8 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * elem)};
  cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)boxh};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, dt == J2D_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base,
                   dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Overlapped covering of [1, n] by windows of `win` cells with a `g`-cell halo:
// returns (start, valid_begin, valid_end) triples; `align` keeps starts ≡ 1 mod align.
static std::vector<int> cover(int n, int win, int g) {
  std::vector<int> out;
  int v = 1;
  while (v <= n) {
    const int s = v == 1 ? 1 : v - g;
    const int e = s + win;  // exclusive
    const int ve = e > n ? n + 1 : e - g;
    out.push_back(s);
    out.push_back(v);
    out.push_back(ve);
    if (ve <= v) break;  // halo too deep for the window
    v = ve;
  }
  return out;
}

// Even covering of [1, n] for the skewed bands: the fewest windows of `win`
// columns (with g-column halos inside) whose valid widths are equal multiples
// of V, so that no band is much narrower than the others (the warps of a
// tile move in lockstep: a narrow band would leave most of a CTA idle while
// its rows still take a full tile's time).  Same triples as cover(); empty
// when a window cannot hold its halos.
static std::vector<int> cover_even(int n, int win, int g, int V) {
  if (n <= win) return {1, 1, n + 1};
  const int cap = win - 2 * g;  // valid width of an inner window
  if (cap < V) return {};
  int m = (n + cap - 1) / cap, wv = 0;
  for (;; ++m) {
    wv = ((n + m - 1) / m + V - 1) / V * V;
    if (wv <= cap) break;
  }
  std::vector<int> out;
  for (int i = 0; i < m; ++i) {
    const int v = 1 + i * wv;
    if (v > n) break;
    out.push_back(i == 0 ? 1 : v - g);
    out.push_back(v);
    out.push_back(std::min(n + 1, v + wv));
  }
  return out;
}

static void ensure(void *&p, size_t &cap, size_t need, cudaError_t &err) {
  if (cap >= need) return;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  err = cudaMalloc(&p, need);
  if (err == cudaSuccess) cap = need;
}

template <typename T>
static void *kernel_ptr(int mode, bool adj, int np) {
  if constexpr (std::is_same<T, float>::value) {
    if (mode == MODE_TILES_PAIR) return (void *)dtb_kernel<float, false, MODE_TILES_PAIR>;
  }
  if (mode == MODE_SKEW) return np == 9 ? (void *)dtb_kernel<T, false, MODE_SKEW, 9> : (void *)dtb_kernel<T, false, MODE_SKEW>;
  if (mode == MODE_GROUPS) return (void *)dtb_kernel<T, false, MODE_GROUPS>;  // batches are forward only
  if (mode == MODE_BANDS) return adj ? (void *)dtb_kernel<T, true, MODE_BANDS> : (void *)dtb_kernel<T, false, MODE_BANDS>;
  return adj ? (void *)dtb_kernel<T, true, MODE_TILES> : (void *)dtb_kernel<T, false, MODE_TILES>;
}

cudaError_t dtb_run(DtbState &S, const DtbRun &r, cudaStream_t s, std::string &err) {
  const auto &grids = *r.grids;
  const j2d_dtype dt = r.dtype;
  const int V = vec_of(dt), SW = 32 * V;
  const size_t elem = dt == J2D_F64 ? 8 : 4;
  const int ctas = r.cfg.ctas;
  // two steps per sweep: FP32 tiles of the forward map
  const bool pair = r.cfg.sweep == 2 && dt == J2D_F32 && r.cfg.algo == J2D_ALGO_TILES && !r.adjoint;
  const bool skew = r.cfg.algo == J2D_ALGO_SKEWED;
  if (skew && r.adjoint) { err = "the skewed schedule is forward only"; return cudaErrorNotSupported; }
  if (grids[0].shape == 9 && (!skew || r.adjoint)) { err = "the box stencil runs the skewed schedule"; return cudaErrorNotSupported; }
  const int rmax = skew ? dtb_rows_max_skew(dt, r.smem_optin)
                        : pair ? dtb_rows_max_pair(dt, r.smem_optin) : dtb_rows_max(dt, r.smem_optin, kWarps);
  const int rp = (rmax + 3) / 4 * 4;
  if (rmax < 2) { err = "shared memory too small"; return cudaErrorNotSupported; }
  const bool single = grids.size() == 1;
  const int mode = skew ? MODE_SKEW
                 : (r.cfg.algo == J2D_ALGO_TILES)                ? MODE_TILES
                 : (r.cfg.algo == J2D_ALGO_RESIDENT && !single) ? MODE_GROUPS
                                                                 : MODE_BANDS;
  if (mode == MODE_BANDS && !single) { err = "bands need a single grid"; return cudaErrorNotSupported; }
  if (mode == MODE_GROUPS && r.adjoint) { err = "batches are forward only"; return cudaErrorNotSupported; }
  if (r.states && (r.adjoint || !single || pair || mode == MODE_SKEW || mode == MODE_GROUPS)) {
    err = "keeping every state needs a forward single-grid run of the single-step strips";
    return cudaErrorNotSupported;
  }

  KParams kp{};
  std::vector<int> jobs, job_off;
  std::vector<long> tkey;
  bool tiles_cached = false;
  int depth = r.cfg.depth, rounds = 1, last = (int)r.steps;
  if (mode == MODE_GROUPS) {
    depth = last = (int)r.steps;
    rounds = 1;
    tkey = {ctas, rmax, (long)grids.size(), 2000};
    for (const GridDesc &g : grids) {
      tkey.push_back(g.nx);
      tkey.push_back(g.ny);
    }
    tiles_cached = tkey == S.tiles_key;
    if (tiles_cached) {
      jobs = S.tiles_jobs;
    } else {
      if (group_waves(grids, SW, ctas, rmax, jobs) == 0) { err = "a grid of the batch does not fit on chip"; return cudaErrorNotSupported; }
      S.tiles_key = tkey;
      S.tiles_jobs = jobs;
      S.tiles_off.clear();
    }
  } else if (r.cfg.algo == J2D_ALGO_RESIDENT) {
    int m = 0;
    if (!resident_fit(grids[0], SW, ctas, rmax, &m)) { err = "grid does not fit on chip"; return cudaErrorNotSupported; }
    kp.bx = choose_bx((grids[0].nx + SW - 1) / SW, grids[0].ny, ctas, &m);
    depth = last = (int)r.steps;
    rounds = 1;
    jobs = {1, grids[0].ny + 1, 1, grids[0].ny + 1, m};
  } else {
    depth = std::max(1, std::min(depth, (int)r.steps));
    rounds = (int)((r.steps + depth - 1) / depth);
    last = (int)(r.steps - (long)(rounds - 1) * depth);
    if (mode == MODE_BANDS) {
      const GridDesc &g = grids[0];
      const int ncs = (g.nx + SW - 1) / SW;
      const long slots = (long)ctas * kWarps;
      if (ncs > slots) { err = "grid too wide for one band"; return cudaErrorNotSupported; }
      int m = 0;
      kp.bx = choose_bx(ncs, g.ny, ctas, &m);
      const int hb = m * rmax;
      auto cv = cover(g.ny, hb, depth);
      if (cv.empty() || cv.back() != g.ny + 1) { err = "band too short for the temporal depth"; return cudaErrorNotSupported; }
      for (size_t i = 0; i + 2 < cv.size(); i += 3) {
        const int bs = cv[i], ve = cv[i + 2];
        const int be = std::min(g.ny + 1, bs + hb);
        const int mm = std::min(m, be - bs);
        jobs.insert(jobs.end(), {bs, be, cv[i + 1], ve, mm});
      }
    } else if (mode == MODE_SKEW) {
      const int wx = r.cfg.tile_wx, wy = kWarps / wx;
      const int tw = wx * SW, th = wy * rmax;
      const int gx = (depth + V - 1) / V * V;
      tkey = {ctas, wx, rmax, depth, (long)grids.size(), 1000};
      for (const GridDesc &g : grids) {
        tkey.push_back(g.nx);
        tkey.push_back(g.ny);
      }
      tiles_cached = tkey == S.tiles_key;
      if (tiles_cached) {
        jobs = S.tiles_jobs;
        job_off = S.tiles_off;
      } else {
        // column bands of every grid (k-deep overlapped halo in x), each
        // carrying the physical rows [1, ny+1) stored at level k
        struct Band { int g, tx0, vx0, vx1, wxa; };
        std::vector<Band> bands;
        long total = 0;
        for (size_t gi = 0; gi < grids.size(); ++gi) {
          const GridDesc &g = grids[gi];
          auto cx = cover_even(g.nx, tw, gx, V);
          if (cx.empty() || cx.back() != g.nx + 1) {
            err = "tile too narrow for the temporal depth";
            return cudaErrorNotSupported;
          }
          for (size_t b = 0; b + 2 < cx.size(); b += 3) {
            int wxa = 0;
            while (wxa < wx && cx[b] + wxa * SW <= g.nx) ++wxa;
            bands.push_back({(int)gi, cx[b], cx[b + 1], cx[b + 2], wxa});
            total += (long)g.ny;
          }
        }
        // split the bands' rows (in band order) into `ctas` runs of equal
        // length (a tile takes the same time whatever its width: its warps
        // move in lockstep); a run is cut into pieces, one per band it touches
        std::vector<std::vector<int>> lists(ctas);
        long acc = 0;
        int cta = 0;
        // A piece of physical rows [v, ve) computes the skewed rows
        // [q0, ve+k): its values at level k are rows v+k .. ve+k-1, and a
        // piece starting inside the band starts 2(k-1) rows before v+k (its
        // top halo is held at level 0).  A last round of fewer steps k' < k
        // runs the same tiles: rows v+k' .. ve+k'-1 lie inside and are clean.
        for (const Band &bd : bands) {
          const GridDesc &g = grids[bd.g];
          const int vend = g.ny + 1;
          int v = 1;
          while (v < vend) {
            const long target = (long)((double)total * (cta + 1) / ctas);
            const long room = target - acc;
            int take = room > 0 ? (int)room : 1;
            take = std::max(take, 4 * depth);  // no pieces much shorter than their overlap
            if (cta == ctas - 1) take = vend - v;
            const int ve = std::min(vend, v + take);
            const int q0 = std::max(1, v + depth - 2 * (depth - 1));
            const int qe = ve + depth;
            for (int q = q0; q < qe; q += th) {
              const int nq = std::min(th, qe - q);
              lists[cta].insert(lists[cta].end(), {bd.g, bd.tx0, bd.vx0, bd.vx1, q, nq, v, ve, q == q0 ? 1 : 0, bd.wxa});
            }
            acc += (long)(ve - v);
            v = ve;
            if (acc >= target && cta < ctas - 1) ++cta;
          }
        }
        job_off.push_back(0);
        for (int b = 0; b < ctas; ++b) {
          jobs.insert(jobs.end(), lists[b].begin(), lists[b].end());
          job_off.push_back((int)(jobs.size() / kSkewInts));
        }
        S.tiles_key = tkey;
        S.tiles_jobs = jobs;
        S.tiles_off = job_off;
      }
    } else {
      const int wx = r.cfg.tile_wx, wy = kWarps / wx;
      const int trows = rmax;
      const int tw = wx * SW, th = wy * trows;
      const int gx = (depth + V - 1) / V * V;
      tkey = {ctas, wx, rmax, depth, (long)grids.size()};
      for (const GridDesc &g : grids) {
        tkey.push_back(g.nx);
        tkey.push_back(g.ny);
      }
      tiles_cached = tkey == S.tiles_key;
      if (tiles_cached) {
        jobs = S.tiles_jobs;
        job_off = S.tiles_off;
      }
      for (size_t gi = 0; gi < grids.size() && !tiles_cached; ++gi) {
        const GridDesc &g = grids[gi];
        // a grid that fits one tile needs no overlapped halo; otherwise the
        // halo of depth k must leave each tile a valid core
        auto cx = cover(g.nx, tw, gx), cy = cover(g.ny, th, depth);
        if (cx.back() != g.nx + 1 || cy.back() != g.ny + 1) {
          err = "tile too small for the temporal depth";
          return cudaErrorNotSupported;
        }
        for (size_t a = 0; a + 2 < cy.size(); a += 3)
          for (size_t b = 0; b + 2 < cx.size(); b += 3) {
            // strips of the tile inside the grid (the rest would idle)
            int wxa = 0, wya = 0;
            while (wxa < wx && cx[b] + wxa * SW <= g.nx) ++wxa;
            while (wya < wy && cy[a] + wya * trows <= g.ny) ++wya;
            jobs.insert(jobs.end(), {(int)gi, cx[b], cy[a], cx[b + 1], cx[b + 2], cy[a + 1], cy[a + 2], 0, wxa, wya, 0});
          }
      }
      kp.tile_rows = trows;
    }
  }
  const int njobs = mode == MODE_GROUPS ? (int)(jobs.size() / ((size_t)ctas * kWarps * kSlotInts))
                                        : (int)(jobs.size() / (mode == MODE_BANDS ? 5 : mode == MODE_SKEW ? kSkewInts : kTileInts));
  // TILES: tiles are packed into groups of at most 16 strips that one CTA runs
  // side by side (a tile keeps only its strips inside the grid, so the small
  // tiles of a batch share CTAs instead of leaving warps idle): largest tiles
  // first, each into the fullest group it fits (best fit).  Groups go to CTAs
  // largest cost (cells) first onto the least-loaded CTA; CTA b runs the
  // tiles [job_off[b], job_off[b+1]), a group's tiles consecutive.
  if (mode == MODE_TILES && !tiles_cached) {
    std::vector<int> order(njobs);
    for (int j = 0; j < njobs; ++j) order[j] = j;
    auto warps_of = [&](int j) { return jobs[(size_t)kTileInts * j + 8] * jobs[(size_t)kTileInts * j + 9]; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return warps_of(x) > warps_of(y); });
    std::vector<std::vector<int>> members;       // tiles of each group
    std::vector<int> used;                       // warps used by each group
    std::vector<std::vector<int>> by_free(kWarps + 1);  // groups by free warps
    for (int j : order) {
      const int n = warps_of(j);
      int gsel = -1;
      for (int f = n; f <= kWarps && gsel < 0; ++f)
        if (!by_free[f].empty()) {
          gsel = by_free[f].back();
          by_free[f].pop_back();
        }
      if (gsel < 0) {
        gsel = (int)members.size();
        members.emplace_back();
        used.push_back(0);
      }
      jobs[(size_t)kTileInts * j + 7] = used[gsel];
      used[gsel] += n;
      members[gsel].push_back(j);
      by_free[kWarps - used[gsel]].push_back(gsel);
    }
    const int ngroups = (int)members.size();
    std::vector<std::pair<long, int>> cost(ngroups);
    for (int gi = 0; gi < ngroups; ++gi) {
      long c = 0;
      for (int j : members[gi]) {
        const int *t = &jobs[(size_t)kTileInts * j];
        const GridDesc &g = grids[t[0]];
        for (int b = 0; b < t[9]; ++b) {
          const int rows = std::min(rmax, g.ny + 1 - (t[2] + b * rmax));
          c += (long)rows * SW * t[8];
        }
      }
      cost[gi] = {c, gi};
    }
    std::stable_sort(cost.begin(), cost.end(), [](const std::pair<long, int> &x, const std::pair<long, int> &y) {
      return x.first > y.first;
    });
    // least-loaded CTA first (ties: lowest index), from a heap
    std::vector<std::vector<int>> lists(ctas);
    std::priority_queue<std::pair<long, int>, std::vector<std::pair<long, int>>, std::greater<std::pair<long, int>>> heap;
    for (int b = 0; b < ctas; ++b) heap.push({0L, b});
    for (const auto &cg : cost) {
      auto top = heap.top();
      heap.pop();
      lists[top.second].push_back(cg.second);
      heap.push({top.first + cg.first, top.second});
    }
    std::vector<int> reordered;
    reordered.reserve(jobs.size());
    job_off.push_back(0);
    for (int b = 0; b < ctas; ++b) {
      for (int gi : lists[b]) {
        const size_t first = reordered.size();
        for (int j : members[gi])
          reordered.insert(reordered.end(), &jobs[(size_t)kTileInts * j], &jobs[(size_t)kTileInts * j] + kTileInts);
        reordered[first + 10] = (int)members[gi].size();
      }
      job_off.push_back((int)(reordered.size() / kTileInts));
    }
    jobs.swap(reordered);
    S.tiles_key = tkey;
    S.tiles_jobs = jobs;
    S.tiles_off = job_off;
  }

  // descriptors: grids, tensor maps, jobs
  const size_t ng = grids.size();
  const size_t off_maps = (ng * sizeof(GridDev) + 127) / 128 * 128;
  const size_t off_jobs = off_maps + ng * 6 * sizeof(CUtensorMap);
  const size_t off_joff = off_jobs + (jobs.size() * sizeof(int) + 15) / 16 * 16;
  const size_t desc_bytes = off_joff + job_off.size() * sizeof(int) + 16;
  std::vector<char> host(desc_bytes, 0);
  GridDev *hg = reinterpret_cast<GridDev *>(host.data());
  CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(host.data() + off_maps);
  bool in_is_out = false;
  for (size_t i = 0; i < ng; ++i) {
    const GridDesc &g = grids[i];
    hg[i].nx = g.nx;
    hg[i].ny = g.ny;
    hg[i].off = (int)g.off;
    hg[i].pitch = g.pitch;
    hg[i].shape = g.shape;
    for (int d = 0; d < 9; ++d) hg[i].w[d] = g.w[d];
    hg[i].buf[0] = const_cast<void *>(r.in[i]);
    hg[i].buf[1] = r.ws[i];
    hg[i].buf[2] = r.out[i];
    if (r.in[i] == r.out[i]) in_is_out = true;
    for (int b = 0; b < 3; ++b) {
      if (!encode_map(&hm[i * 6 + b], dt, hg[i].buf[b], g.pitch, g.off + g.nx + 2, g.ny + 2, SW, rmax) ||
          !encode_map(&hm[i * 6 + 3 + b], dt, hg[i].buf[b], g.pitch, g.off + g.nx + 1, g.ny + 1, SW, 1)) {
        err = "cuTensorMapEncodeTiled failed";
        return cudaErrorNotSupported;
      }
    }
  }
  memcpy(host.data() + off_jobs, jobs.data(), jobs.size() * sizeof(int));
  if (!job_off.empty()) memcpy(host.data() + off_joff, job_off.data(), job_off.size() * sizeof(int));
  cudaError_t e = cudaSuccess;
  ensure(S.desc, S.desc_bytes, desc_bytes, e);
  if (e != cudaSuccess) { err = "descriptor allocation"; return cudaErrorMemoryAllocation; }
  const size_t slot_bytes = (size_t)WarpLayout<double>::mailbox_elems(rp) * 8;  // sized for the larger type
  const size_t nslots = (size_t)ctas * kWarps;
  // SKEWED: per CTA, two parities x (k+1) levels x two rows x the band width
  const size_t skew_tw = mode == MODE_SKEW ? (size_t)r.cfg.tile_wx * SW : 0;
  const size_t skew_bytes = mode == MODE_SKEW ? (size_t)ctas * 2 * (depth + 1) * 2 * skew_tw * elem : 0;
  const size_t skew_off = (256 + nslots * sizeof(int) + 255) / 256 * 256;
  const size_t scratch = mode == MODE_SKEW ? skew_off + skew_bytes
                                           : 256 + nslots * sizeof(int) +
                                                 (mode == MODE_BANDS || mode == MODE_GROUPS ? nslots * slot_bytes : 0);
  ensure(S.scratch, S.scratch_bytes, scratch, e);
  if (e != cudaSuccess) { err = "scratch allocation"; return cudaErrorMemoryAllocation; }
  // upload the descriptors unless the device copy already holds them (a run
  // repeated on the same buffers uploads nothing, so it can be captured into
  // a CUDA graph after one plain run)
  if (S.last_desc != host) {
    if ((e = cudaMemcpyAsync(S.desc, host.data(), desc_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
      err = "descriptor upload";
      return e;
    }
    S.last_desc = host;
  }
  char *sc = (char *)S.scratch;
  if ((e = cudaMemsetAsync(sc, 0, 256, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc + 256, 0xff, nslots * sizeof(int), s)) != cudaSuccess) {
    err = "scratch reset";
    return e;
  }

  // the global range this launch may touch (grid buffers, scratch,
  // descriptors): the checked build tests every global access against it
  unsigned long long mem_lo = ~0ull, mem_hi = 0;
  auto span = [&](const void *b, size_t n) {
    mem_lo = std::min(mem_lo, (unsigned long long)b);
    mem_hi = std::max(mem_hi, (unsigned long long)b + n);
  };
  for (size_t i = 0; i < ng; ++i)
    for (int b = 0; b < 3; ++b) span(hg[i].buf[b], grids[i].bytes(elem));
  span(S.scratch, scratch);
  span(S.desc, desc_bytes);
  if (r.states) span(r.states, (size_t)r.steps * (size_t)r.state_elems * elem);
  kp.mem_lo = mem_lo;
  kp.mem_hi = mem_hi;

  // ring of every buffer a round writes = ring of the input (constant forward;
  // corners and the starting values of the adjoint ring accumulation)
  int src0 = 0;
  {
    const GridDev *gd = reinterpret_cast<const GridDev *>(S.desc);
    note_launch();
    if (dt == J2D_F64)
      ring_copy_grids_kernel<double><<<dim3((unsigned)ng, 2), 256, 0, s>>>(gd, rounds > 1, 1, mem_lo, mem_hi);
    else
      ring_copy_grids_kernel<float><<<dim3((unsigned)ng, 2), 256, 0, s>>>(gd, rounds > 1, 1, mem_lo, mem_hi);
    if ((e = cudaGetLastError()) != cudaSuccess) { err = "ring copy"; return e; }
  }
  // overlapped halos read neighbours' cells: a round must not write its source
  const int dst0 = ((rounds - 1) & 1) == 0 ? 2 : 1;
  if (in_is_out && dst0 == 2 && r.cfg.algo != J2D_ALGO_RESIDENT) {
    for (size_t i = 0; i < ng; ++i)
      if ((e = cudaMemcpyAsync(r.ws[i], r.in[i], grids[i].bytes(elem), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    src0 = 1;
  }

  kp.grids = reinterpret_cast<const GridDev *>(S.desc);
  kp.maps = reinterpret_cast<const CUtensorMap *>((char *)S.desc + off_maps);
  kp.jobs = reinterpret_cast<const int *>((char *)S.desc + off_jobs);
  kp.job_off = reinterpret_cast<const int *>((char *)S.desc + off_joff);
  kp.njobs = njobs;
  kp.rounds = rounds;
  kp.depth = depth;
  kp.last_depth = last;
  kp.src0 = src0;
  kp.rmax = rmax;
  kp.rp = rp;
  kp.status = r.status;
  kp.barrier = reinterpret_cast<int *>(sc);
  kp.gflags = reinterpret_cast<int *>(sc + 256);
  kp.gslots = sc + 256 + nslots * sizeof(int);
  kp.timeout_ns = r.timeout_ns;
  // fault injection mutes a strip with a neighbour in another CTA: the first
  // slot when slots run down the columns, else the last column of the first
  // CTA block
  kp.mute_slot = r.mute_slot < 0 ? -1 : (kp.bx > 0 ? kp.bx - 1 : 0);
  kp.int_path = r.int_path;
  kp.states = r.states;
  kp.state_elems = r.state_elems;
  kp.dead_all = 0;
  if (mode == MODE_BANDS || mode == MODE_GROUPS)
    for (const GridDesc &g : grids) kp.dead_all |= g.nx % SW != 0;
  if (mode == MODE_SKEW) {
    kp.skewbuf = sc + skew_off;
    kp.skew_tw = (int)skew_tw;
    kp.skew_levels = depth + 1;
    kp.skew_wx = r.cfg.tile_wx;
  }

  const size_t smem = skew ? skew_smem_bytes((int)elem, rmax)
                           : pair ? pair_smem_bytes((int)elem, rmax) : dtb_smem_bytes((int)elem, rmax, rp);
  const int kmode = pair ? MODE_TILES_PAIR : mode;
  void *fn = dt == J2D_F64 ? kernel_ptr<double>(kmode, r.adjoint, grids[0].shape)
                           : kernel_ptr<float>(kmode, r.adjoint, grids[0].shape);
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
    err = "shared memory attribute";
    return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void *args[] = {&kp};
  note_launch();
  if (r.ev0) cudaEventRecord(r.ev0, s);
  e = cudaLaunchKernelExC(&cfg, fn, args);
  if (e != cudaSuccess) {
    err = "cooperative launch";
    return e;
  }
  if (r.ev1) cudaEventRecord(r.ev1, s);
  return e;
}

int dtb_bounds_fault() {
#ifdef J2D_BOUNDS_CHECK
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_fault, sizeof v) != cudaSuccess) return 0;
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_bounds_fault, &z, sizeof z);
  }
  return v;
#else
  return 0;
#endif
}

void dtb_release(DtbState &S) {
  cudaFree(S.scratch);
  cudaFree(S.desc);
  S = DtbState{};
}

void dtb_invalidate(DtbState &S) { S.last_desc.clear(); }

}  // namespace j2d
