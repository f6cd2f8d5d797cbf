// stream.cu -- temporal blocking in the register file: the STREAM schedule.
//
// The paper's deep temporal blocking (Zhang et al., GPGPU'23, Sections 3.1 and
// 3.3, Figure 1) keeps a tile on chip for several time steps so that one trip
// through HBM carries many steps.  On GB300 the register file (256 KB per SM)
// is larger than shared memory (228 KB), so this schedule keeps the time steps
// of a tile in registers; shared memory only stages the input rows on their
// way in (a ring of a few rows per warp, filled by asynchronous copies).
//
// Each warp owns one column band of the grid, 32 lanes x one 16-byte vector
// (128 FP32 / 64 FP64 columns), and a run of rows, and sweeps the run from top
// to bottom once per pass.  A pass advances M time steps as a pipeline: when
// row i of the pass's input arrives, the warp evaluates step 1 of row i-1,
// step 2 of row i-2, ..., step M of row i-M, each from the two rows of the step
// below that it keeps in registers and the row that step has just produced
// (the update of row r at step t reads rows r-1, r and r+1 of step t-1).  Row
// i-M at step M leaves for HBM.  The x +- 1 neighbours come from the adjacent
// lanes by shuffles; beyond the warp's two edges the missing neighbours spoil
// one more column per step, so a band evaluates 32V columns and stores the
// middle 32V - 2G (G >= M, a multiple of V): an overlapped halo in x, as the
// paper's tiles have.  In y, a run starts M rows above its first stored row
// and ends M rows below its last, so the runs of a band overlap by 2M rows.
// The ring (one cell deep, held constant) is kept by holding a ring cell's
// value at every step: ring columns in the bands that contain one (a select
// per cell), ring rows in the few iterations of a run where a step reaches row
// 0 or row ny+1 (a uniform test).  Cells outside the logical array never
// reach a stored cell: the held ring separates them.
//
// Every cell is evaluated exactly as the one-step kernel evaluates it: FP32 by
// the chain of stencil() in common.cuh (here two cells per paired FP32 multiply
// and fused multiply-add, each element rounded as the scalar instruction
// rounds it), FP64 by stencil_cell() with the integer path on the same cells.
// So the results are bit-identical to every other kernel of the library.
//
// One launch per pass (the passes of a run are ordered on the stream; a run of
// S steps is ceil(S / M) passes, the first one taking the remainder), with
// several waves of (band, run) units so that the block scheduler balances the
// SMs.  Per cell update HBM carries 2 * sizeof(T) * (1 + overlap) / M bytes.
// The same pipeline serves the 3x3 box (j2d9pt) and, for state-keeping runs,
// stores every step's rows instead of the last step's only.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace j2d {

// Warps per block (each warp is independent): FP32 one, so that registers
// are granted warp by warp (FP32 16384^2, k = 8: 3808 against 3228 GCells/s
// with four-warp blocks); FP64 four (155.6 against 161.2 with one).
template <typename T> struct WarpsOf { static constexpr int W = 1; };
template <> struct WarpsOf<double> { static constexpr int W = 4; };
inline int stream_warps(j2d_dtype dt) { return dt == J2D_F64 ? WarpsOf<double>::W : WarpsOf<float>::W; }

struct StreamParams {
  const void *in;
  void *out;
  long pitch;   // elements per row
  int off;      // element offset of logical column 0
  int nx, ny;
  int G;        // halo columns on each side of a band (a multiple of V, >= the pass's steps)
  int vw;       // stored (valid) columns per band: 32V - 2G
  int bands;    // column bands
  int H;        // rows stored per run
  int runs;     // runs per band
  int meff;     // steps of this pass (<= M: steps t > meff leave rows unchanged)
  void *keep;   // keeping every state: step t's rows go to keep + (t - 1) * keep_stride
  long keep_stride;
  int ipath;    // FP64: integer path on
  long nelem;   // elements of each buffer ((ny + 2) * pitch), for the checked build
  int *status;  // checked build: J2D_ERR_BOUNDS is recorded here
  double w[9];  // five-point: W, E, S, C, N; box: the nine weights, rows y-1, y, y+1, columns x-1, x, x+1
};

// ---- one lane's 16-byte vector of a row, in registers -------------------------

// FP32: four columns v0..v3 held as two pairs a = (v0, v2), b = (v1, v3), so
// that the x - 1 and x + 1 operands of each pair are pairs too (mostly the
// other pair), and one paired instruction evaluates two cells.
struct RowF {
  float2 a, b;
};
struct WeightsF {
  float2 w, e, s, c, n;  // each weight in both halves
};

__device__ __forceinline__ RowF row_zero(RowF *) { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ void row_store(float *p, const RowF &r) {
  *reinterpret_cast<float4 *>(p) = make_float4(r.a.x, r.b.x, r.a.y, r.b.y);
}
// Keep the cells whose bit is set in m (bit v: column v of the vector) at c.
__device__ __forceinline__ RowF row_hold(RowF n, const RowF &c, unsigned m) {
  if (m & 1u) n.a.x = c.a.x;
  if (m & 2u) n.b.x = c.b.x;
  if (m & 4u) n.a.y = c.a.y;
  if (m & 8u) n.b.y = c.b.y;
  return n;
}

// One step of the four cells of row c (ym: the row above at the same step,
// yp: the row below), in the order of stencil(): y-1, centre, x-1, x+1, y+1.
// The two operand pairs that would mix registers of both pairs (x-1 of
// (v0, v2) is (L, v1); x+1 of (v1, v3) is (v2, R)) take two scalar FMAs each
// instead of a move into a register pair and one paired FMA.
__device__ __forceinline__ RowF row_step(const WeightsF &k, const RowF &ym, const RowF &c, const RowF &yp) {
  const float L = __shfl_up_sync(0xffffffffu, c.b.y, 1);    // column x0 - 1: the left lane's v3
  const float R = __shfl_down_sync(0xffffffffu, c.a.x, 1);  // column x0 + 4: the right lane's v0
  float2 ra = __fmul2_rn(k.s, ym.a);
  ra = __ffma2_rn(k.c, c.a, ra);
  ra.x = __fmaf_rn(k.w.x, L, ra.x);      // x-1 of v0
  ra.y = __fmaf_rn(k.w.x, c.b.x, ra.y);  // x-1 of v2
  ra = __ffma2_rn(k.e, c.b, ra);         // x+1 of (v0, v2)
  ra = __ffma2_rn(k.n, yp.a, ra);
  float2 rb = __fmul2_rn(k.s, ym.b);
  rb = __ffma2_rn(k.c, c.b, rb);
  rb = __ffma2_rn(k.w, c.a, rb);         // x-1 of (v1, v3)
  rb.x = __fmaf_rn(k.e.x, c.a.y, rb.x);  // x+1 of v1
  rb.y = __fmaf_rn(k.e.x, R, rb.y);      // x+1 of v3
  rb = __ffma2_rn(k.n, yp.b, rb);
  return {ra, rb};
}

// FP64: two columns.
struct RowD {
  double a, b;
};
struct WeightsD {
  Links<double> l;
  ExactW u;
};

__device__ __forceinline__ RowD row_zero(RowD *) { return {0.0, 0.0}; }
__device__ __forceinline__ void row_store(double *p, const RowD &r) {
  *reinterpret_cast<double2 *>(p) = make_double2(r.a, r.b);
}
__device__ __forceinline__ RowD row_hold(RowD n, const RowD &c, unsigned m) {
  if (m & 1u) n.a = c.a;
  if (m & 2u) n.b = c.b;
  return n;
}
// ea, eb: the row's two cells take the integer path (exact_cell(): the same
// cells as in every other kernel).
__device__ __forceinline__ RowD row_step(const WeightsD &k, const RowD &ym, const RowD &c, const RowD &yp,
                                         bool ea, bool eb) {
  const double L = __shfl_up_sync(0xffffffffu, c.b, 1);
  const double R = __shfl_down_sync(0xffffffffu, c.a, 1);
  return {stencil_cell(k.l, k.u, ea, L, c.b, ym.a, c.a, yp.a), stencil_cell(k.l, k.u, eb, c.a, R, ym.b, c.b, yp.b)};
}

// ---- the 3x3 box (j2d9pt): every row also carries its outer neighbours ---------
// A box cell reads the x - 1 and x + 1 columns of all three rows, so a row's
// two values beyond the lane (L: column x0 - 1, R: the column after the
// lane's last) are taken by shuffles once, when the row is produced, and
// travel with it through the three steps that read it.  The chain order is
// that of stencil_box() in common.cuh.
struct RowF9 {
  float2 a, b;  // (v0, v2), (v1, v3) as in RowF
  float L, R;
};
struct WeightsF9 {
  float2 w[9];  // Box9 chain order, each weight in both halves
};
struct RowD9 {
  double a, b, L, R;
};
struct WeightsD9 {
  Box9<double> b;
  ExactWN<9> u;
};

__device__ __forceinline__ RowF9 row_zero(RowF9 *) { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f, 0.f}; }
__device__ __forceinline__ RowD9 row_zero(RowD9 *) { return {0.0, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ void row_nbrs(RowF9 &r) {
  r.L = __shfl_up_sync(0xffffffffu, r.b.y, 1);
  r.R = __shfl_down_sync(0xffffffffu, r.a.x, 1);
}
__device__ __forceinline__ void row_nbrs(RowD9 &r) {
  r.L = __shfl_up_sync(0xffffffffu, r.b, 1);
  r.R = __shfl_down_sync(0xffffffffu, r.a, 1);
}
__device__ __forceinline__ void row_store(float *p, const RowF9 &r) {
  *reinterpret_cast<float4 *>(p) = make_float4(r.a.x, r.b.x, r.a.y, r.b.y);
}
__device__ __forceinline__ void row_store(double *p, const RowD9 &r) {
  *reinterpret_cast<double2 *>(p) = make_double2(r.a, r.b);
}
__device__ __forceinline__ RowF9 row_hold(RowF9 n, const RowF9 &c, unsigned m) {
  if (m & 1u) n.a.x = c.a.x;
  if (m & 2u) n.b.x = c.b.x;
  if (m & 4u) n.a.y = c.a.y;
  if (m & 8u) n.b.y = c.b.y;
  return n;
}
__device__ __forceinline__ RowD9 row_hold(RowD9 n, const RowD9 &c, unsigned m) {
  if (m & 1u) n.a = c.a;
  if (m & 2u) n.b = c.b;
  return n;
}

// Terms in chain order: (y-1, x), (y-1, x-1), (y-1, x+1), (y, x), (y, x-1),
// (y, x+1), (y+1, x), (y+1, x-1), (y+1, x+1).  For the pair (v0, v2) the
// x - 1 operands (L, v1) mix the pairs and take scalar FMAs, the x + 1
// operands are the pair (v1, v3); for (v1, v3) the x - 1 operands are
// (v0, v2) and the x + 1 operands (v2, R) take scalar FMAs.
__device__ __forceinline__ RowF9 row_step9(const WeightsF9 &k, const RowF9 &ym, const RowF9 &c, const RowF9 &yp) {
  float2 ra = __fmul2_rn(k.w[0], ym.a);
  ra.x = __fmaf_rn(k.w[1].x, ym.L, ra.x);
  ra.y = __fmaf_rn(k.w[1].x, ym.b.x, ra.y);
  ra = __ffma2_rn(k.w[2], ym.b, ra);
  ra = __ffma2_rn(k.w[3], c.a, ra);
  ra.x = __fmaf_rn(k.w[4].x, c.L, ra.x);
  ra.y = __fmaf_rn(k.w[4].x, c.b.x, ra.y);
  ra = __ffma2_rn(k.w[5], c.b, ra);
  ra = __ffma2_rn(k.w[6], yp.a, ra);
  ra.x = __fmaf_rn(k.w[7].x, yp.L, ra.x);
  ra.y = __fmaf_rn(k.w[7].x, yp.b.x, ra.y);
  ra = __ffma2_rn(k.w[8], yp.b, ra);
  float2 rb = __fmul2_rn(k.w[0], ym.b);
  rb = __ffma2_rn(k.w[1], ym.a, rb);
  rb.x = __fmaf_rn(k.w[2].x, ym.a.y, rb.x);
  rb.y = __fmaf_rn(k.w[2].x, ym.R, rb.y);
  rb = __ffma2_rn(k.w[3], c.b, rb);
  rb = __ffma2_rn(k.w[4], c.a, rb);
  rb.x = __fmaf_rn(k.w[5].x, c.a.y, rb.x);
  rb.y = __fmaf_rn(k.w[5].x, c.R, rb.y);
  rb = __ffma2_rn(k.w[6], yp.b, rb);
  rb = __ffma2_rn(k.w[7], yp.a, rb);
  rb.x = __fmaf_rn(k.w[8].x, yp.a.y, rb.x);
  rb.y = __fmaf_rn(k.w[8].x, yp.R, rb.y);
  return {ra, rb, 0.f, 0.f};
}
__device__ __forceinline__ RowD9 row_step9(const WeightsD9 &k, const RowD9 &ym, const RowD9 &c, const RowD9 &yp,
                                           bool ea, bool eb) {
  return {stencil_box_cell(k.b, k.u, ea, ym.L, ym.a, ym.b, c.L, c.a, c.b, yp.L, yp.a, yp.b),
          stencil_box_cell(k.b, k.u, eb, ym.a, ym.b, ym.R, c.a, c.b, c.R, yp.a, yp.b, yp.R), 0.0, 0.0};
}

template <typename T, int SH> struct RowOf;
template <> struct RowOf<float, 5> { using R = RowF; using W = WeightsF; };
template <> struct RowOf<double, 5> { using R = RowD; using W = WeightsD; };
template <> struct RowOf<float, 9> { using R = RowF9; using W = WeightsF9; };
template <> struct RowOf<double, 9> { using R = RowD9; using W = WeightsD9; };

// Five-point rows take their neighbours when they are read.
__device__ __forceinline__ void row_nbrs(RowF &) {}
__device__ __forceinline__ void row_nbrs(RowD &) {}

// ea, eb: the lane's first / second cell takes the integer path (FP64; known
// at compile time where the trip's row phases are: the column parities of a
// lane's two cells are fixed, its first column being odd).
__device__ __forceinline__ RowF step_any(const WeightsF &k, const RowF &ym, const RowF &c, const RowF &yp, bool,
                                         bool) {
  return row_step(k, ym, c, yp);
}
__device__ __forceinline__ RowD step_any(const WeightsD &k, const RowD &ym, const RowD &c, const RowD &yp, bool ea,
                                         bool eb) {
  return row_step(k, ym, c, yp, ea, eb);
}
__device__ __forceinline__ RowF9 step_any(const WeightsF9 &k, const RowF9 &ym, const RowF9 &c, const RowF9 &yp, bool,
                                          bool) {
  return row_step9(k, ym, c, yp);
}
__device__ __forceinline__ RowD9 step_any(const WeightsD9 &k, const RowD9 &ym, const RowD9 &c, const RowD9 &yp,
                                          bool ea, bool eb) {
  return row_step9(k, ym, c, yp, ea, eb);
}

// In the checked build, is [e, e + V) inside the buffer of nelem elements?
__device__ __forceinline__ bool stream_ok(long e, int V, const StreamParams &p) {
  if (!kChecked) return true;
  const bool ok = e >= 0 && e + V <= p.nelem;
  if (!ok) set_error(p.status, DEV_BOUNDS);
  return ok;
}

// The pipeline of one warp: for each step t = 0..M-1 the two most recent rows
// of step t (A: the older, B: the newer).
// KEEP: every step's rows are stored (to p.keep), not only the last step's.
template <typename T, int M, bool EDGE, bool IP, bool KEEP, int SH> struct Pipe {
  using R = typename RowOf<T, SH>::R;
  using W = typename RowOf<T, SH>::W;
  R A[M], B[M];
  const W &k;
  const StreamParams &p;
  T *out;
  long e0;        // element offset of this lane's vector within a row
  int x0;         // logical column of the vector's first element
  unsigned hold;  // ring columns in this lane's vector
  bool st;        // this lane's vector is stored
  int y0, y1;     // stored rows [y0, y1)

  __device__ __forceinline__ Pipe(const W &k_, const StreamParams &p_, T *out_, long e0_, int x0_, unsigned hold_,
                                  bool st_, int y0_, int y1_)
      : k(k_), p(p_), out(out_), e0(e0_), x0(x0_), hold(hold_), st(st_), y0(y0_), y1(y1_) {
#pragma unroll
    for (int t = 0; t < M; ++t) {
      A[t] = row_zero((R *)nullptr);
      B[t] = row_zero((R *)nullptr);
    }
  }

  // Iteration i: row i of step 0 arrives; steps 1..M advance one row each.
  // CHK: some step reaches ring row 0 or ny + 1 in this iteration, or the
  // pass has fewer than M steps (steps beyond meff pass their rows through).
  // ph: i mod 4 when the caller knows it at compile time (FP64 trips), so
  // that each step's integer-path choice (exact_cell(): rows y mod 4 in
  // {0, 1}) is a constant; -1 otherwise.
  template <bool CHK> __device__ __forceinline__ void iter(int i, R cur, int ph) {
#pragma unroll
    for (int t = 1; t <= M; ++t) {
      const int r = i - t;  // the row step t evaluates
      const int yy = ph >= 0 ? ph - t + 4 * M : r;  // the row, or a row of the same phase mod 4
      R n = step_any(k, A[t - 1], B[t - 1], cur, IP && exact_cell(1, yy, true), IP && exact_cell(0, yy, true));
      if (EDGE) n = row_hold(n, B[t - 1], hold);
      if (CHK && (r == 0 || r == p.ny + 1 || t > p.meff)) n = B[t - 1];
      if (SH == 9 && t < M) row_nbrs(n);  // read with its neighbours by steps t + 1 (three times)
      A[t - 1] = B[t - 1];
      B[t - 1] = cur;
      cur = n;
      if (KEEP && t <= p.meff && st && r >= y0 && r < y1) {
        const long e = (long)r * p.pitch + e0;
        if (stream_ok(e, VecOf<T>::V, p)) row_store(static_cast<T *>(p.keep) + (t - 1) * p.keep_stride + e, n);
      }
    }
    const int r = i - M;
    if (!KEEP && st && r >= y0 && r < y1) {
      const long e = (long)r * p.pitch + e0;
      if (stream_ok(e, VecOf<T>::V, p)) row_store(out + e, cur);
    }
  }
};

// Input rows reach the warp through a ring of shared-memory slots of one row
// each (16 bytes per lane), filled by asynchronous copies kAhead rows ahead of
// use: the copies wait in the memory system instead of in registers.  Each
// lane copies and reads back only its own 16 bytes, so the ring needs no
// synchronisation beyond the lane's own copy groups.  The ring has two trips'
// worth of slots (2U >= kAhead + 2), so a slot is refilled at least two
// iterations after it was read.
constexpr int kAhead = 4;

// Iterations per trip of the sweep loop.  FP32: 3, the period of a step's
// three-row window, so the unrolled trip rotates its registers without moves.
// FP64: 4, the period of the integer-path row pattern (trips start on rows 0
// mod 4, so each step's choice between the integer path and the FMA chain is
// known at compile time and the trip is straight-line code).
template <typename T> struct TripOf { static constexpr int U = 3; };
template <> struct TripOf<double> { static constexpr int U = 4; };
constexpr int kStageMax = 8;  // slots per warp, the largest 2U

__device__ __forceinline__ void stage_copy(uint32_t dst, const void *src, bool on) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(on ? 16 : 0) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 1) : "memory"); }
__device__ __forceinline__ void stage_drain() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Start the copy of input row i into the slot at shared address dst (rows
// past the ring row ny + 1, and vectors outside the row, read as zero).
template <typename T>
__device__ __forceinline__ void issue_row(const T *in, const StreamParams &p, int i, long e0, bool live, uint32_t dst) {
  bool on = live && i <= p.ny + 1;
  const long e = on ? (long)i * p.pitch + e0 : 0;
  if (on) on = stream_ok(e, VecOf<T>::V, p);
  stage_copy(dst, in + (on ? e : 0), on);
}

__device__ __forceinline__ RowF read_slot(const float4 *q, RowF *) {
  const float4 v = *q;
  return {make_float2(v.x, v.z), make_float2(v.y, v.w)};
}
__device__ __forceinline__ RowF9 read_slot(const float4 *q, RowF9 *) {
  const float4 v = *q;
  RowF9 r = {make_float2(v.x, v.z), make_float2(v.y, v.w), 0.f, 0.f};
  row_nbrs(r);
  return r;
}
__device__ __forceinline__ RowD9 read_slot(const float4 *q, RowD9 *) {
  const double2 v = *reinterpret_cast<const double2 *>(q);
  RowD9 r = {v.x, v.y, 0.0, 0.0};
  row_nbrs(r);
  return r;
}
__device__ __forceinline__ RowD read_slot(const float4 *q, RowD *) {
  const double2 v = *reinterpret_cast<const double2 *>(q);
  return {v.x, v.y};
}

template <typename T, int M, bool EDGE, bool IP, bool KEEP, int SH>
__device__ __forceinline__ void stream_sweep(const StreamParams &p, const typename RowOf<T, SH>::W &k, long e0, int x0,
                                             unsigned hold, bool live, bool st, int y0, int y1, float4 *ring) {
  using R = typename RowOf<T, SH>::R;
  constexpr int U = TripOf<T>::U;
  constexpr int S = 2 * U;  // slots
  static_assert(S >= kAhead + 2 && S <= kStageMax, "ring too small");
  const T *in = static_cast<const T *>(p.in);
  T *out = static_cast<T *>(p.out);
  Pipe<T, M, EDGE, IP, KEEP, SH> pipe(k, p, out, e0, x0, hold, st, y0, y1);
  int a = max(y0 - M, 0);  // earlier rows only warm the pipeline up
  if (U == 4) a &= ~3;
  const int iend = y1 + M;  // the last iteration stores row y1 - 1
  const bool short_pass = p.meff < M;
  // this lane's slot j is ring[32 * j]; row a + n sits in slot n mod S
  const uint32_t base = smem_u32(ring);
#pragma unroll
  for (int j = 0; j < kAhead; ++j) issue_row(in, p, a + j, e0, live, base + 512u * j);
  int s = 0;  // slot of row i: 0 or U
  for (int i = a; i < iend; i += U) {
    if (short_pass || i <= M || i + U - 1 >= p.ny + 2) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        stage_wait();
        const R c = read_slot(ring + 32 * (s + u), (R *)nullptr);
        const int sn = s + u + kAhead;
        issue_row(in, p, i + u + kAhead, e0, live, base + 512u * (sn >= S ? sn - S : sn));
        pipe.template iter<true>(i + u, c, U == 4 ? u : -1);
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        stage_wait();
        const R c = read_slot(ring + 32 * (s + u), (R *)nullptr);
        const int sn = s + u + kAhead;
        issue_row(in, p, i + u + kAhead, e0, live, base + 512u * (sn >= S ? sn - S : sn));
        pipe.template iter<false>(i + u, c, U == 4 ? u : -1);
      }
    }
    s = s == 0 ? U : 0;
  }
  stage_drain();
}

__device__ __forceinline__ void make_weights(const StreamParams &p, WeightsF *k) {
  const float w = (float)p.w[0], e = (float)p.w[1], s = (float)p.w[2], c = (float)p.w[3], n = (float)p.w[4];
  k->w = make_float2(w, w);
  k->e = make_float2(e, e);
  k->s = make_float2(s, s);
  k->c = make_float2(c, c);
  k->n = make_float2(n, n);
}
__device__ __forceinline__ void make_weights(const StreamParams &p, WeightsF9 *k) {
  const Box9<float> b = box_chain<float>(p.w);
#pragma unroll
  for (int i = 0; i < 9; ++i) k->w[i] = make_float2(b.w[i], b.w[i]);
}
__device__ __forceinline__ void make_weights(const StreamParams &p, WeightsD9 *k) {
  k->b = box_chain<double>(p.w);
  k->u = box_exact_weights(k->b);
}
__device__ __forceinline__ void make_weights(const StreamParams &p, WeightsD *k) {
  k->l = Links<double>{p.w[0], p.w[1], p.w[2], p.w[3], p.w[4]};
  k->u = exact_weights(k->l);
}

template <typename T, int M, bool IP, bool KEEP, int SH>
__global__ void __launch_bounds__(32 * WarpsOf<T>::W) stream_kernel(StreamParams p) {
  constexpr int V = VecOf<T>::V;
  const int lane = threadIdx.x & 31;
  const int unit = blockIdx.x * WarpsOf<T>::W + (threadIdx.x >> 5);
  if (unit >= p.bands * p.runs) return;  // whole warps
  // units in band-fastest order: the warps running at the same time cover
  // neighbouring bands of the same rows, so the overlapped halo columns two
  // bands read are found in L2 the second time
  const int band = unit % p.bands, run = unit / p.bands;
  const int xb = 1 + band * p.vw - p.G;  // logical column of lane 0's first element
  const int x0 = xb + V * lane;
  const long e0 = p.off + x0;
  const bool live = e0 >= 0 && e0 + V <= p.pitch;
  const bool st = live && x0 >= xb + p.G && x0 < xb + 32 * V - p.G && x0 <= p.nx;
  unsigned hold = 0;
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (x0 + v == 0 || x0 + v == p.nx + 1) hold |= 1u << v;
  const bool edge = __any_sync(0xffffffffu, hold != 0);
  const int y0 = 1 + run * p.H, y1 = min(y0 + p.H, p.ny + 1);
  typename RowOf<T, SH>::W k;
  make_weights(p, &k);
  __shared__ float4 ring[WarpsOf<T>::W][2 * TripOf<T>::U * 32];
  float4 *mine = &ring[threadIdx.x >> 5][lane];
  if (edge)
    stream_sweep<T, M, true, IP, KEEP, SH>(p, k, e0, x0, hold, live, st, y0, y1, mine);
  else
    stream_sweep<T, M, false, IP, KEEP, SH>(p, k, e0, x0, hold, live, st, y0, y1, mine);
}

// ---- host side ------------------------------------------------------------------

using StreamFn = void (*)(StreamParams);

template <typename T, bool IP, bool KEEP, int SH, int... Ms> struct StreamTable;
template <typename T, bool IP, bool KEEP, int SH> struct StreamTable<T, IP, KEEP, SH> {
  static StreamFn get(int) { return nullptr; }
};
template <typename T, bool IP, bool KEEP, int SH, int M0, int... Ms> struct StreamTable<T, IP, KEEP, SH, M0, Ms...> {
  static StreamFn get(int m) {
    return m == M0 ? stream_kernel<T, M0, IP, KEEP, SH> : StreamTable<T, IP, KEEP, SH, Ms...>::get(m);
  }
};

int stream_max_depth(j2d_dtype dt) { return dt == J2D_F64 ? kStreamMaxF64 : kStreamMaxF32; }

// Steps per pass with a kernel of their own; a run's shorter pass runs the
// kernel of the run's depth with fewer steps.  Runs that keep every state
// have kernels for fewer depths.
static StreamFn stream_fn(j2d_dtype dt, int m, int ipath, bool keep = false, int shape = 5) {
  if (shape == 9) {  // the box: no state-keeping runs
    if (keep) return nullptr;
    if (dt == J2D_F64)
      return ipath ? StreamTable<double, true, false, 9, 2, 3, 4>::get(m)
                   : StreamTable<double, false, false, 9, 2, 3, 4>::get(m);
    return StreamTable<float, false, false, 9, 4, 6, 8>::get(m);
  }
  if (dt == J2D_F64) {
    if (keep)
      return ipath ? StreamTable<double, true, true, 5, 2, 3, 4>::get(m)
                   : StreamTable<double, false, true, 5, 2, 3, 4>::get(m);
    return ipath ? StreamTable<double, true, false, 5, 2, 3, 4, 6>::get(m)
                 : StreamTable<double, false, false, 5, 2, 3, 4, 6>::get(m);
  }
  if (keep) return StreamTable<float, false, true, 5, 4, 8>::get(m);
  return StreamTable<float, false, false, 5, 4, 6, 8, 10, 12>::get(m);
}

bool stream_depth_ok(j2d_dtype dt, int m, int shape) { return stream_fn(dt, m, 1, false, shape) != nullptr; }
bool stream_keep_ok(j2d_dtype dt, int m) { return stream_fn(dt, m, 1, true) != nullptr; }

// Resident blocks per SM of one instantiation (cached).
static int stream_occupancy(j2d_dtype dt, int m, int shape) {
  static std::mutex mu;
  static int cache[2][2][16] = {};
  std::lock_guard<std::mutex> lk(mu);
  int &c = cache[shape == 9 ? 1 : 0][dt == J2D_F64 ? 1 : 0][m];
  if (c == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stream_fn(dt, m, 1, false, shape), 32 * stream_warps(dt), 0) != cudaSuccess ||
        nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    c = nb;
  }
  return c;
}

StreamGeom stream_geometry(j2d_dtype dt, const GridDesc &g, int depth, int sms) {
  const int d = std::max(1, std::min(depth, stream_max_depth(dt)));
  const long warps = (long)stream_occupancy(dt, d, g.shape) * stream_warps(dt) * std::max(sms, 1);
  return stream_geometry_warps(dt, g.nx, g.ny, depth, warps);
}

StreamGeom stream_geometry_warps(j2d_dtype dt, int nx, int ny, int depth, long warps) {
  StreamGeom q;
  const int V = dt == J2D_F64 ? 2 : 4;
  q.depth = std::max(1, std::min(depth, stream_max_depth(dt)));
  q.G = (q.depth + V - 1) / V * V;
  q.vw = 32 * V - 2 * q.G;
  q.bands = (nx + q.vw - 1) / q.vw;
  // Several waves of units per pass, so that the block scheduler balances
  // the SMs as units finish (FP64 k = 2 on 16384^2: 159 GCells/s with one
  // wave of units, 178 / 191 / 194 / 189 / 175 with 2 / 4 / 8 / 16 / 32;
  // FP32 k = 8: 3958, 4254 with 2 or 3, 4235 with 4, 4090 with 8), each run
  // at least 32M (FP64) or 16M (FP32) rows tall, its 2M-row overlap then
  // costing at most 6% or 12% (FP64 8192^2: 169.7 GCells/s against 164.8 with
  // 16M; FP32 4096^2: 2764 against 2175 with 32M).
  warps = std::max(warps, 1L);
  const int waves = dt == J2D_F64 ? 8 : 3;
  const int hmin = (dt == J2D_F64 ? 32 : 16) * q.depth;
  int runs = (int)std::max<long>(1, waves * warps / q.bands);
  runs = std::min(runs, std::max(1, ny / hmin));
  q.H = (ny + runs - 1) / runs;
  q.runs = (ny + q.H - 1) / q.H;
  return q;
}

// A pass of m <= q.depth steps, in -> out (distinct buffers whose rings
// agree); with keep set, step t's state goes to keep + (t - 1) * keep_stride
// elements instead (out unused).
cudaError_t launch_stream_pass(j2d_dtype dt, const void *in, void *out, const GridDesc &g, const StreamGeom &q, int m,
                               int ipath, int *status, cudaStream_t s, void *keep, long keep_stride) {
  StreamParams p;
  p.in = in;
  p.out = out;
  p.pitch = g.pitch;
  p.off = (int)g.off;
  p.nx = g.nx;
  p.ny = g.ny;
  p.G = q.G;
  p.vw = q.vw;
  p.bands = q.bands;
  p.H = q.H;
  p.runs = q.runs;
  p.meff = m;
  p.keep = keep;
  p.keep_stride = keep_stride;
  p.ipath = ipath;
  p.nelem = (long)(g.ny + 2) * g.pitch;
  p.status = status;
  for (int i = 0; i < 9; ++i) p.w[i] = g.w[i];
  StreamFn fn = stream_fn(dt, q.depth, ipath, keep != nullptr, g.shape);
  if (!fn || m < 1 || m > q.depth) return cudaErrorInvalidValue;
  const long units = (long)q.bands * q.runs;
  const int W = stream_warps(dt);
  const unsigned blocks = (unsigned)((units + W - 1) / W);
  fn<<<blocks, 32 * W, 0, s>>>(p);
  note_launch();
  return cudaGetLastError();
}

}  // namespace j2d
