// dtb.h -- host interface of the temporally blocked kernels (dtb.cu).
#pragma once

#include <string>
#include <vector>

#include "internal.h"

struct j2d5pt_plan_s;

namespace j2d {

struct DtbRequest {
  int algo = J2D_ALGO_AUTO;
  int depth = 0;
  int tile_wx = 0;
  int ctas = 0;
  long steps = 0;
  bool adjoint = false;
  int sweep_steps = 2;  // TILES, FP32 forward: steps per sweep (J2D_OPT_SWEEP_STEPS)
};

// Everything one temporally blocked run needs.
struct DtbRun {
  j2d_dtype dtype = J2D_F64;
  const std::vector<GridDesc> *grids = nullptr;
  const void *const *in = nullptr;
  void *const *out = nullptr;
  void **ws = nullptr;
  long steps = 0;
  bool adjoint = false;
  DtbConfig cfg;
  int *status = nullptr;
  unsigned long long timeout_ns = 0;
  int sms = 0;
  size_t smem_optin = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // recorded around the kernel if set
  int mute_slot = -1;                         // fault injection (J2D_OPT_FAULT_INJECT): >= 0 = on
  int int_path = 0;                           // FP64 integer path on (J2D_OPT_INT_PATH)
  void *states = nullptr;                     // keep every state: state t+1 at states + t * state_elems (forward,
  long state_elems = 0;                       // one grid, RESIDENT / BANDS / single-step TILES)
};

// Device scratch and cached launch data owned by a plan.
struct DtbState {
  void *scratch = nullptr;  // barrier counter, flags, halo mailboxes
  size_t scratch_bytes = 0;
  void *desc = nullptr;     // grid descriptors, tensor maps, job lists
  size_t desc_bytes = 0;
  std::vector<char> last_desc;  // host copy of what `desc` holds
  // TILES job lists of the last run, reused while their key (CTAs, tile
  // shape, rows, depth, grid sizes) is unchanged
  std::vector<long> tiles_key;
  std::vector<int> tiles_jobs, tiles_off;
};

// Largest rows per warp strip that fit in shared memory.
int dtb_rows_max(j2d_dtype dt, size_t smem_optin, int warps);
// The same for the two-steps-per-sweep tiles (no mailboxes; at most 32 rows).
int dtb_rows_max_pair(j2d_dtype dt, size_t smem_optin);
// The same for the skewed tiles (no mailboxes; at most 32 rows).
int dtb_rows_max_skew(j2d_dtype dt, size_t smem_optin);

DtbConfig dtb_choose(j2d_dtype dt, const std::vector<GridDesc> &grids, int sms, size_t smem_optin,
                     const DtbRequest &rq);
cudaError_t dtb_run(DtbState &st, const DtbRun &r, cudaStream_t s, std::string &err);
void dtb_release(DtbState &st);
// Checked build: J2D_ERR_BOUNDS if a bound test failed since the last call
// (and clears it); 0 otherwise, and always 0 in the regular build.
int dtb_bounds_fault();
void dtb_invalidate(DtbState &st);  // forget the uploaded descriptors (weights changed)

}  // namespace j2d
