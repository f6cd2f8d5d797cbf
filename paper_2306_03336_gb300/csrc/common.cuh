// common.cuh -- device helpers shared by the j2d5pt kernels (sm_103a).
//
// The stencil (Zhang et al., GPGPU'23, Section 3.1, Listing 1) updates a cell
// from its x-1, x+1, y-1, centre and y+1 neighbours with weights W, E, S, C, N.
// Every kernel here evaluates a cell the same way: the chain of one product
// and four fused multiply-adds (stencil() below) or, for the FP64 cells the
// integer path selects, the correctly rounded exact sum (stencil_exact()).  So
// the one-step kernel and the temporally blocked kernels give bit-identical
// results for the same inputs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace j2d {

// Device-side status codes (mirrors of j2d_status values).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 6, DEV_BOUNDS = 7 };

// Elements per 16-byte vector: 2 doubles or 4 floats.
template <typename T> struct VecOf;
template <> struct VecOf<double> { static constexpr int V = 2; using type = double2; };
template <> struct VecOf<float> { static constexpr int V = 4; using type = float4; };

// The five link weights of one cell: x-1, x+1, y-1, centre, y+1.
template <typename T> struct Links { T xm, xp, ym, c, yp; };

// Base weights as the user gives them: W (x-1), E (x+1), S (y-1), C, N (y+1).
template <typename T> struct Weights { T w[5]; };

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// One cell update: the product of the y-1 link, then fused multiply-adds of
// the centre, x-1, x+1 and y+1 links.  The order starts with the operands a
// row sweep already holds in registers and ends with the ones that arrive
// last (lane shuffles, the next row), so the chain does not wait on them.
// Every kernel uses this one order: results are bit-identical across kernels.
template <typename T>
__device__ __forceinline__ T stencil(const Links<T> &a, T xm, T xp, T ym, T c, T yp) {
  T r = mul_rn(a.ym, ym);
  r = fma_rn(a.c, c, r);
  r = fma_rn(a.xm, xm, r);
  r = fma_rn(a.xp, xp, r);
  r = fma_rn(a.yp, yp, r);
  return r;
}

// ---- FP64 cells evaluated on the integer pipes -------------------------------
// GB300 retires two FP64 FMAs per clock per SM, so an FP64 stencil saturates
// that pipe while the integer pipes idle.  A fixed subset of FP64 cells is
// therefore evaluated without the FP64 pipe: the update becomes the correctly
// rounded (round-to-nearest-even) value of the exact five-term sum, computed in
// 32/64-bit integer arithmetic.  It is an FP64 result at least as accurate as
// the FMA chain (one rounding instead of five).  Which cells take this path
// depends only on the cell's logical coordinates (kExactMask, when the run has
// the path on), and the fast path's own fallback to
// stencil() only on the cell's inputs, so every kernel still produces the same
// bits for the same cell.
//
// Fast path: all five weights and values positive normal, exponent spread of
// the five products at most kExactGuard bits, normal result; otherwise the
// cell takes the FMA chain.  Exactness: each value's 53-bit significand is
// shifted left by its product's place in the frame, s <= kExactGuard = 11
// bits (so it still fits 64 bits), and multiplied by the weight's 53-bit
// significand: each term has at most 117 bits, five of them sum without loss
// in a 128-bit frame (< 5 * 2^117 < 2^120), so the frame holds the exact sum
// and one rounding gives the correctly rounded value.  (A guard of 11 rather
// than a wider one saves two shifts per term, the value being shifted before
// the multiply instead of the 106-bit product after it.)
// bit (y & 3) * 2 + (x & 1) set: cell (x, y) takes the integer path.  Rows
// with y mod 4 in {0, 1}: half of the cells, the pattern that measured fastest
// across the resident, tiles and one-step kernels.
constexpr unsigned kExactMask = 0x0F;
constexpr int kExactGuard = 11;

// Weight significands and exponents of an NT-term cell for the integer path.
template <int NT> struct ExactWN {
  uint64_t m[NT];  // significands with the implicit bit, in the cell's term order
  int e[NT];       // biased exponents
  bool ok;         // all NT positive normal
};
using ExactW = ExactWN<5>;  // the five-point cell: order xm, xp, ym, c, yp

template <int NT> __device__ __forceinline__ ExactWN<NT> exact_weights_n(const double (&w)[NT]) {
  ExactWN<NT> u;
  u.ok = true;
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    const uint64_t b = (uint64_t)__double_as_longlong(w[i]);
    u.e[i] = (int)(b >> 52);  // includes the sign bit: negative weights fail the range test
    u.ok &= (unsigned)(u.e[i] - 1) < 2046u;
    u.m[i] = (b & ((1ull << 52) - 1)) | (1ull << 52);
  }
  return u;
}

__device__ __forceinline__ ExactW exact_weights(const Links<double> &a) {
  const double w[5] = {a.xm, a.xp, a.ym, a.c, a.yp};
  return exact_weights_n<5>(w);
}

// Four-word (128-bit) add with carry: a += b.
__device__ __forceinline__ void add128(uint32_t (&a)[4], uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
      : "r"(b0), "r"(b1), "r"(b2), "r"(b3));
}

// Correctly rounded sum of the NT products w[i] * v[i] on the fast path;
// returns false (r untouched) when the fast path does not apply.
// Significands are split into 32-bit words (high word 21 bits with the
// implicit bit); a product of the shifted value significand (two words) and
// the weight significand is four 32x32->64 multiplies; the frame is four
// 32-bit words.  Each term is below 2^(64+53) = 2^117, so up to 2^11 terms
// fit the 128-bit frame without loss (NT = 5: the frame stays below 2^120;
// NT = 9: below 2^121).
template <int NT>
__device__ __forceinline__ bool stencil_exact_n(const ExactWN<NT> &u, const double (&v)[NT], double &r) {
  uint32_t m0[NT], m1[NT];
  int E[NT];
  bool ok = true;
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    const uint32_t hi = (uint32_t)__double2hiint(v[i]);
    m0[i] = (uint32_t)__double2loint(v[i]);
    const int e = (int)(hi >> 20);  // includes the sign bit: negative values fail the range test
    ok &= (unsigned)(e - 1) < 2046u;
    m1[i] = (hi & 0xFFFFFu) | 0x100000u;
    E[i] = e + u.e[i];  // product i = p_i * 2^(E[i] - 2150), p_i in [2^104, 2^106)
  }
  int Em = E[0];
#pragma unroll
  for (int i = 1; i < NT; ++i) Em = max(Em, E[i]);
  uint32_t f[4] = {0u, 0u, 0u, 0u};
  int sall = 0;
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    const int s = kExactGuard - (Em - E[i]);  // frame position: p_i * 2^s, s <= kExactGuard
    sall |= s;                               // any s < 0 leaves the fast path
    const uint32_t a0 = m0[i] << (s & 31), a1 = __funnelshift_l(m0[i], m1[i], s);  // value significand * 2^s
    const uint32_t b0 = (uint32_t)u.m[i], b1 = (uint32_t)(u.m[i] >> 32);
    const uint64_t p00 = (uint64_t)a0 * b0;
    const uint64_t p01 = (uint64_t)a0 * b1 + (p00 >> 32);
    const uint64_t p10 = (uint64_t)a1 * b0 + (uint32_t)p01;
    const uint64_t p11 = (uint64_t)a1 * b1 + (p01 >> 32) + (p10 >> 32);
    add128(f, (uint32_t)p00, (uint32_t)p10, (uint32_t)p11, (uint32_t)(p11 >> 32));
  }
  ok &= sall >= 0;
  // frame F = f[3]:f[2]:f[1]:f[0] = sum * 2^(2150 + kExactGuard - Em), F in [2^115, 2^121)
  const int z = __clz((int)f[3]) & 31;  // 7..12 on the fast path
  const uint32_t g3 = __funnelshift_l(f[2], f[3], z), g2 = __funnelshift_l(f[1], f[2], z);
  const uint32_t g1 = __funnelshift_l(f[0], f[1], z), g0 = f[0] << z;
  uint64_t kept = ((uint64_t)g3 << 21) | (g2 >> 11);  // the top 53 bits
  const uint64_t rb = (g2 >> 10) & 1u;
  const bool sticky = ((g2 & 0x3FFu) | g1 | g0) != 0u;
  kept += rb & ((uint64_t)sticky | (kept & 1u));
  const int carry = (int)(kept >> 53) & 1;  // kept <= 2^53 on the fast path
  kept >>= carry;
  const int e = Em - 1000 - kExactGuard - z + carry;  // biased exponent of the result
  ok &= (unsigned)(e - 1) < 2046u;
  if (ok) r = __longlong_as_double((long long)(((uint64_t)(e - 1) << 52) + kept));
  return ok;
}

// The five-point cell: xm*W + xp*E + ym*S + c*C + yp*N.
__device__ __forceinline__ bool stencil_exact(const ExactW &u, double xm, double xp, double ym, double c, double yp,
                                              double &r) {
  const double v[5] = {xm, xp, ym, c, yp};
  return stencil_exact_n<5>(u, v, r);
}

// Whether cell (x, y) takes the integer path (logical coordinates) in a run
// with the path on.  The pattern is a compile-time constant, so this reduces
// to a test of y.
__device__ __forceinline__ bool exact_cell(int x, int y, bool on) {
  return on && ((kExactMask >> (((y & 3) << 1) | (x & 1))) & 1u);
}

// stencil() or, for the cells exact_cell() selects, the integer path.
__device__ __forceinline__ double stencil_cell(const Links<double> &a, const ExactW &u, bool exact, double xm,
                                               double xp, double ym, double c, double yp) {
  double r;
  if (exact && u.ok && stencil_exact(u, xm, xp, ym, c, yp, r)) return r;
  return stencil(a, xm, xp, ym, c, yp);
}

// ---- the 3x3 box stencil (j2d9pt) --------------------------------------------
// A second stencil shape through the same kernels.  Weights come in the
// user's order (rows y-1, y, y+1, columns x-1, x, x+1); every box kernel
// evaluates a cell as the product of the (y-1, x) term, then fused
// multiply-adds of (y-1, x-1), (y-1, x+1), (y, x), (y, x-1), (y, x+1),
// (y+1, x), (y+1, x-1), (y+1, x+1): the operands of the row a sweep loads
// last enter last.  Box9 holds the weights in that chain order.
template <typename T> struct Box9 { T w[9]; };

// The chain over three rows (m: y-1, c: y, p: y+1), each as (x-1, x, x+1).
template <typename T>
__device__ __forceinline__ T stencil_box(const Box9<T> &b, T m0, T m1, T m2, T c0, T c1, T c2, T p0, T p1, T p2) {
  T r = mul_rn(b.w[0], m1);
  r = fma_rn(b.w[1], m0, r);
  r = fma_rn(b.w[2], m2, r);
  r = fma_rn(b.w[3], c1, r);
  r = fma_rn(b.w[4], c0, r);
  r = fma_rn(b.w[5], c2, r);
  r = fma_rn(b.w[6], p1, r);
  r = fma_rn(b.w[7], p0, r);
  r = fma_rn(b.w[8], p2, r);
  return r;
}

// FP64: the integer path on the cells exact_cell() selects, else the chain.
__device__ __forceinline__ double stencil_box_cell(const Box9<double> &b, const ExactWN<9> &u, bool exact,
                                                   double m0, double m1, double m2, double c0, double c1, double c2,
                                                   double p0, double p1, double p2) {
  double r;
  if (exact && u.ok) {
    const double v[9] = {m1, m0, m2, c1, c0, c2, p1, p0, p2};  // chain order, as the weights
    if (stencil_exact_n<9>(u, v, r)) return r;
  }
  return stencil_box(b, m0, m1, m2, c0, c1, c2, p0, p1, p2);
}
__device__ __forceinline__ float stencil_box_cell(const Box9<float> &b, const ExactWN<9> &, bool, float m0, float m1,
                                                  float m2, float c0, float c1, float c2, float p0, float p1,
                                                  float p2) {
  return stencil_box(b, m0, m1, m2, c0, c1, c2, p0, p1, p2);
}

// Box weights in chain order from the user's order.
template <typename T> __host__ __device__ inline Box9<T> box_chain(const double *w) {
  return Box9<T>{{(T)w[1], (T)w[0], (T)w[2], (T)w[4], (T)w[3], (T)w[5], (T)w[7], (T)w[6], (T)w[8]}};
}
__device__ __forceinline__ ExactWN<9> box_exact_weights(const Box9<double> &b) { return exact_weights_n<9>(b.w); }

// Link weights of logical cell (x, y) of an nx*ny grid with a one-cell ring.
// Forward: interior cells use W, E, S, C, N; ring and outside cells keep their
// value (identity).  Adjoint (the transpose of one forward step): interior
// cells use the mirrored weights with links to ring cells removed; a ring cell
// keeps its value and adds its one interior neighbour times the weight of
// the forward link that read it; corners and outside cells keep their value.
template <typename T, bool ADJ>
__device__ __forceinline__ Links<T> cell_links(int x, int y, int nx, int ny, const Weights<T> &w) {
  const T W = w.w[0], E = w.w[1], S = w.w[2], C = w.w[3], N = w.w[4];
  const T z = T(0), one = T(1);
  const bool xi = (x >= 1) && (x <= nx), yi = (y >= 1) && (y <= ny);
  if (!ADJ) {
    if (xi && yi) return {W, E, S, C, N};
    return {z, z, z, one, z};
  }
  if (xi && yi) return {x >= 2 ? E : z, x <= nx - 1 ? W : z, y >= 2 ? N : z, C, y <= ny - 1 ? S : z};
  if (yi && x == 0) return {z, W, z, one, z};
  if (yi && x == nx + 1) return {E, z, z, one, z};
  if (xi && y == 0) return {z, z, z, one, S};
  if (xi && y == ny + 1) return {z, z, N, one, z};
  return {z, z, z, one, z};
}

// ---- small PTX wrappers ----------------------------------------------------

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(int *p, int v) {
  asm volatile("st.relaxed.gpu.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_cta(int *p, int v) {
  asm volatile("st.relaxed.cta.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_acq_rel_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }

// Global loads that bypass L1 (halo mailboxes written by other SMs).
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory vector / scalar access on 32-bit shared addresses.  volatile:
// kept in program order with the other shared-memory accesses of the warp
// (the strip is updated in place).
template <typename T> __device__ __forceinline__ void lds_v(uint32_t a, T *o);
template <> __device__ __forceinline__ void lds_v<double>(uint32_t a, double *o) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(o[0]), "=d"(o[1]) : "r"(a) : "memory");
}
template <> __device__ __forceinline__ void lds_v<float>(uint32_t a, float *o) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(a) : "memory");
}
template <typename T> __device__ __forceinline__ void sts_v(uint32_t a, const T *o);
template <> __device__ __forceinline__ void sts_v<double>(uint32_t a, const double *o) {
  asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(o[0]), "d"(o[1]) : "memory");
}
template <> __device__ __forceinline__ void sts_v<float>(uint32_t a, const float *o) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]) : "memory");
}
template <typename T> __device__ __forceinline__ T lds_s(uint32_t a);
template <> __device__ __forceinline__ double lds_s<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
template <> __device__ __forceinline__ float lds_s<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

// mbarrier (shared memory transaction barrier) for TMA completion.
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

// 2D tiled TMA load: box at (x, y) of the tensor map into shared memory,
// completing on `bar` with the box's byte count.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const void *tmap, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Hint: bring a 2D tile of global memory into L2 ahead of its load (no
// completion to wait for, no shared memory touched).
__device__ __forceinline__ void tma_prefetch_2d(const void *tmap, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tmap), "r"(x), "r"(y)
               : "memory");
}
// 2D tiled TMA store from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, const void *smem_src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap),
               "r"(x), "r"(y), "r"(smem_u32(smem_src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// ---- the checked build (-DJ2D_BOUNDS_CHECK) --------------------------------------
// The blocked kernels reach shared and global memory through ldm / stm / vload /
// vstore (dtb.cu).  In the checked build every such access is tested first: a
// shared address against the launch's dynamic shared memory, a global address
// against the range of the buffers the launch may touch (set at kernel start);
// a failed test records J2D_ERR_BOUNDS (reported by j2d5pt_sync_status) and the
// access is skipped (a load reads zero).  The regular build compiles the tests
// away: kChecked is false and the accessors are plain loads and stores.
#ifdef J2D_BOUNDS_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool smem_window_ok(const void *p, unsigned bytes) {
  extern __shared__ char j2d_dynamic_smem[];
  unsigned size;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
  const uint32_t a = smem_u32(p), b = smem_u32(j2d_dynamic_smem);
  return a >= b && a + bytes <= b + size;
}

// Record the first device-side error of a run; later errors are dropped.
__device__ __forceinline__ void set_error(int *status, int code) {
  if (status) atomicCAS(status, DEV_OK, code);
}
__device__ __forceinline__ bool has_error(const int *status) {
  return status && *((volatile const int *)status) != DEV_OK;
}

}  // namespace j2d
