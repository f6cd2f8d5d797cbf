/*
 * j2d5pt_oracle.c -- plain CPU oracle for the 2D Jacobi 5-point stencil (j2d5pt).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
 * that the CUDA library is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library never does.
 * It shares no code, header or constant with the CUDA path.
 *
 * What it computes (Zhang et al., "Exploiting Scratchpad Memory for Deep
 * Temporal Blocking", GPGPU'23, Section 3.1, Listing 1):
 *   out[y][x] = W*in[y][x-1] + E*in[y][x+1] + S*in[y-1][x] + C*in[y][x] + N*in[y+1][x]
 * evaluated out of place (Jacobi: separate input and output arrays), for every
 * interior cell 1<=x<=nx, 1<=y<=ny, summed left to right in exactly that order,
 * in IEEE binary64 with round-to-nearest and no fused multiply-add (this file
 * must be compiled with -ffp-contract=off).  The paper is silent on the
 * boundary; the reading used here is a one-cell Dirichlet ring that is held
 * constant: ring cells of `out` equal those of `in`.
 *
 * Arrays are dense, row-major, (ny+2) rows of (nx+2) values, x fastest; row 0
 * and row ny+1, column 0 and column nx+1 are the ring.  Weights are {W,E,S,C,N}.
 *
 * The time loop (Section 3.1: the time loop moved inside the kernel; Section
 * 3.3: tiles advanced several steps at a time) does not change the result,
 * so the oracle for every tiling and temporal depth is the same plain
 * iteration below.
 *
 * Adjoint and weight gradient (not in the paper; they follow from the forward
 * map by linear algebra): one step is u' = M u with M = [[A_II, A_IR],[0, I]]
 * over (interior, ring) cells.  The adjoint step is lam = M^T lam', computed
 * here literally as the transpose: every interior cell scatters its value,
 * times the weight of each of its five links, onto the cell that link reads;
 * ring cells also keep their own value (the identity block).  The weight
 * gradient of L = <g, u_T> is dL/dw_d = sum_t sum_i lam_{t+1}[i] * u_t[nbr_d(i)].
 */
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(y, x) ((size_t)(y) * (size_t)(nx + 2) + (size_t)(x))

/* One forward step (Listing 1 arithmetic, fixed left-to-right order). */
static void step_rows(int nx, int ny, const double *w, const double *in, double *out,
                      int nthreads) {
  const double W = w[0], E = w[1], S = w[2], C = w[3], N = w[4];
  int y;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (y = 1; y <= ny; ++y) {
    for (int x = 1; x <= nx; ++x) {
      double acc = W * in[IDX(y, x - 1)];
      acc = acc + E * in[IDX(y, x + 1)];
      acc = acc + S * in[IDX(y - 1, x)];
      acc = acc + C * in[IDX(y, x)];
      acc = acc + N * in[IDX(y + 1, x)];
      out[IDX(y, x)] = acc;
    }
  }
  (void)nthreads;
  /* Dirichlet ring: held constant. */
  for (int x = 0; x < nx + 2; ++x) {
    out[IDX(0, x)] = in[IDX(0, x)];
    out[IDX(ny + 1, x)] = in[IDX(ny + 1, x)];
  }
  for (int yy = 1; yy <= ny; ++yy) {
    out[IDX(yy, 0)] = in[IDX(yy, 0)];
    out[IDX(yy, nx + 1)] = in[IDX(yy, nx + 1)];
  }
}

void oracle_j2d5pt_step(int nx, int ny, const double *w, const double *in, double *out) {
  step_rows(nx, ny, w, in, out, 1);
}

/* `steps` forward steps; u0 -> uT.  Uses one scratch array, ping-pong. */
int oracle_j2d5pt_run(int nx, int ny, const double *w, const double *u0, double *uT,
                      long steps, int nthreads) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  double *a = (double *)malloc(n * sizeof(double));
  double *b = (double *)malloc(n * sizeof(double));
  if (!a || !b) { free(a); free(b); return 1; }
  memcpy(a, u0, n * sizeof(double));
  for (long t = 0; t < steps; ++t) {
    step_rows(nx, ny, w, a, b, nthreads);
    double *tmp = a; a = b; b = tmp;
  }
  memcpy(uT, a, n * sizeof(double));
  free(a);
  free(b);
  return 0;
}

/* Same iteration in binary32 storage and arithmetic (weights rounded to
 * float), for the single-precision form; also no FMA. */
int oracle_j2d5pt_run_f32(int nx, int ny, const float *w, const float *u0, float *uT,
                          long steps, int nthreads) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  float *a = (float *)malloc(n * sizeof(float));
  float *b = (float *)malloc(n * sizeof(float));
  if (!a || !b) { free(a); free(b); return 1; }
  memcpy(a, u0, n * sizeof(float));
  const float W = w[0], E = w[1], S = w[2], C = w[3], N = w[4];
  for (long t = 0; t < steps; ++t) {
    int y;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (y = 1; y <= ny; ++y) {
      for (int x = 1; x <= nx; ++x) {
        float acc = W * a[IDX(y, x - 1)];
        acc = acc + E * a[IDX(y, x + 1)];
        acc = acc + S * a[IDX(y - 1, x)];
        acc = acc + C * a[IDX(y, x)];
        acc = acc + N * a[IDX(y + 1, x)];
        b[IDX(y, x)] = acc;
      }
    }
    for (int x = 0; x < nx + 2; ++x) {
      b[IDX(0, x)] = a[IDX(0, x)];
      b[IDX(ny + 1, x)] = a[IDX(ny + 1, x)];
    }
    for (int yy = 1; yy <= ny; ++yy) {
      b[IDX(yy, 0)] = a[IDX(yy, 0)];
      b[IDX(yy, nx + 1)] = a[IDX(yy, nx + 1)];
    }
    float *tmp = a; a = b; b = tmp;
  }
  memcpy(uT, a, n * sizeof(float));
  free(a);
  free(b);
  (void)nthreads;
  return 0;
}

/* One adjoint step lam = M^T lam1, written as the literal transpose of the
 * forward step: start from the identity block on the ring (ring cells keep
 * their value, interior cells start at zero), then let every interior cell i
 * add w_d * lam1[i] onto the cell its link d reads. */
void oracle_j2d5pt_adjoint_step(int nx, int ny, const double *w, const double *lam1,
                                double *lam) {
  const double W = w[0], E = w[1], S = w[2], C = w[3], N = w[4];
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  for (size_t i = 0; i < n; ++i) lam[i] = 0.0;
  for (int x = 0; x < nx + 2; ++x) {
    lam[IDX(0, x)] = lam1[IDX(0, x)];
    lam[IDX(ny + 1, x)] = lam1[IDX(ny + 1, x)];
  }
  for (int y = 1; y <= ny; ++y) {
    lam[IDX(y, 0)] = lam1[IDX(y, 0)];
    lam[IDX(y, nx + 1)] = lam1[IDX(y, nx + 1)];
  }
  for (int y = 1; y <= ny; ++y) {
    for (int x = 1; x <= nx; ++x) {
      double g = lam1[IDX(y, x)];
      lam[IDX(y, x - 1)] += W * g;
      lam[IDX(y, x + 1)] += E * g;
      lam[IDX(y - 1, x)] += S * g;
      lam[IDX(y, x)] += C * g;
      lam[IDX(y + 1, x)] += N * g;
    }
  }
}

int oracle_j2d5pt_adjoint_run(int nx, int ny, const double *w, const double *lamT,
                              double *lam0, long steps) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  double *a = (double *)malloc(n * sizeof(double));
  double *b = (double *)malloc(n * sizeof(double));
  if (!a || !b) { free(a); free(b); return 1; }
  memcpy(a, lamT, n * sizeof(double));
  for (long t = 0; t < steps; ++t) {
    oracle_j2d5pt_adjoint_step(nx, ny, w, a, b);
    double *tmp = a; a = b; b = tmp;
  }
  memcpy(lam0, a, n * sizeof(double));
  free(a);
  free(b);
  return 0;
}

/* Neumaier's compensated summation (Neumaier 1974): sum and running correction. */
typedef struct { double s, c; } csum;
static void csum_add(csum *k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}

/* dw[d] += sum over interior i of lam1[i] * u[nbr_d(i)], d in {W,E,S,C,N}:
 * the derivative of <lam1, M(w) u> with respect to each weight. */
void oracle_j2d5pt_weight_grad(int nx, int ny, const double *u, const double *lam1,
                               double *dw) {
  csum k[5];
  for (int d = 0; d < 5; ++d) { k[d].s = dw[d]; k[d].c = 0.0; }
  for (int y = 1; y <= ny; ++y) {
    for (int x = 1; x <= nx; ++x) {
      double g = lam1[IDX(y, x)];
      csum_add(&k[0], g * u[IDX(y, x - 1)]);
      csum_add(&k[1], g * u[IDX(y, x + 1)]);
      csum_add(&k[2], g * u[IDX(y - 1, x)]);
      csum_add(&k[3], g * u[IDX(y, x)]);
      csum_add(&k[4], g * u[IDX(y + 1, x)]);
    }
  }
  for (int d = 0; d < 5; ++d) dw[d] = k[d].s + k[d].c;
}

/* <a, b> over all (ny+2)(nx+2) cells, compensated. */
double oracle_dot(int nx, int ny, const double *a, const double *b) {
  csum k = {0.0, 0.0};
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  for (size_t i = 0; i < n; ++i) csum_add(&k, a[i] * b[i]);
  return k.s + k.c;
}

/* Full reverse sweep for L = <g, u_T>: gradient with respect to u0 (lam0) and
 * to the five weights (dw), storing the whole forward trajectory.  Small
 * problems only; it is the plain definition the checkpointed GPU path is
 * checked against. */
int oracle_j2d5pt_grad(int nx, int ny, const double *w, const double *u0, const double *g,
                       long steps, double *lam0, double *dw) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  double *traj = (double *)malloc(n * sizeof(double) * (size_t)(steps + 1));
  double *lam = (double *)malloc(n * sizeof(double));
  double *tmp = (double *)malloc(n * sizeof(double));
  if (!traj || !lam || !tmp) { free(traj); free(lam); free(tmp); return 1; }
  memcpy(traj, u0, n * sizeof(double));
  for (long t = 0; t < steps; ++t) oracle_j2d5pt_step(nx, ny, w, traj + n * t, traj + n * (t + 1));
  for (int d = 0; d < 5; ++d) dw[d] = 0.0;
  memcpy(lam, g, n * sizeof(double));
  for (long t = steps - 1; t >= 0; --t) {
    oracle_j2d5pt_weight_grad(nx, ny, traj + n * t, lam, dw);
    oracle_j2d5pt_adjoint_step(nx, ny, w, lam, tmp);
    memcpy(lam, tmp, n * sizeof(double));
  }
  memcpy(lam0, lam, n * sizeof(double));
  free(traj);
  free(lam);
  free(tmp);
  return 0;
}

/* ---- j2d9pt: the nine-point box stencil -------------------------------------
 *
 * The paper presents j2d5pt as a case study of deep temporal blocking (title,
 * Section 1); its step function (Section 3.1) does not depend on the shape of
 * the stencil.  The second shape built here is the 3x3 box:
 *   out[y][x] = sum over dy = -1, 0, 1 and dx = -1, 0, 1 of
 *               w[3*(dy+1) + (dx+1)] * in[y+dy][x+dx]
 * i.e. weights in the order (y-1: x-1, x, x+1), (y: x-1, x, x+1),
 * (y+1: x-1, x, x+1), the y-1 row first as the paper's S link reads the row
 * below.  Summed left to right in that order, binary64, no fused
 * multiply-add, out of place; the one-cell ring is held constant. */
static void box_rows(int nx, int ny, const double *w, const double *in, double *out, int nthreads) {
  int y;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (y = 1; y <= ny; ++y) {
    for (int x = 1; x <= nx; ++x) {
      double acc = w[0] * in[IDX(y - 1, x - 1)];
      acc = acc + w[1] * in[IDX(y - 1, x)];
      acc = acc + w[2] * in[IDX(y - 1, x + 1)];
      acc = acc + w[3] * in[IDX(y, x - 1)];
      acc = acc + w[4] * in[IDX(y, x)];
      acc = acc + w[5] * in[IDX(y, x + 1)];
      acc = acc + w[6] * in[IDX(y + 1, x - 1)];
      acc = acc + w[7] * in[IDX(y + 1, x)];
      acc = acc + w[8] * in[IDX(y + 1, x + 1)];
      out[IDX(y, x)] = acc;
    }
  }
  (void)nthreads;
  for (int x = 0; x < nx + 2; ++x) {
    out[IDX(0, x)] = in[IDX(0, x)];
    out[IDX(ny + 1, x)] = in[IDX(ny + 1, x)];
  }
  for (int yy = 1; yy <= ny; ++yy) {
    out[IDX(yy, 0)] = in[IDX(yy, 0)];
    out[IDX(yy, nx + 1)] = in[IDX(yy, nx + 1)];
  }
}

void oracle_j2d9pt_step(int nx, int ny, const double *w, const double *in, double *out) {
  box_rows(nx, ny, w, in, out, 1);
}

int oracle_j2d9pt_run(int nx, int ny, const double *w, const double *u0, double *uT, long steps, int nthreads) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  double *a = (double *)malloc(n * sizeof(double));
  double *b = (double *)malloc(n * sizeof(double));
  if (!a || !b) { free(a); free(b); return 1; }
  memcpy(a, u0, n * sizeof(double));
  for (long t = 0; t < steps; ++t) {
    box_rows(nx, ny, w, a, b, nthreads);
    double *tmp = a; a = b; b = tmp;
  }
  memcpy(uT, a, n * sizeof(double));
  free(a);
  free(b);
  return 0;
}

/* The same iteration in binary32 storage and arithmetic (weights rounded to
 * float), no FMA. */
int oracle_j2d9pt_run_f32(int nx, int ny, const float *w, const float *u0, float *uT, long steps, int nthreads) {
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  float *a = (float *)malloc(n * sizeof(float));
  float *b = (float *)malloc(n * sizeof(float));
  if (!a || !b) { free(a); free(b); return 1; }
  memcpy(a, u0, n * sizeof(float));
  for (long t = 0; t < steps; ++t) {
    int y;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (y = 1; y <= ny; ++y) {
      for (int x = 1; x <= nx; ++x) {
        float acc = w[0] * a[IDX(y - 1, x - 1)];
        acc = acc + w[1] * a[IDX(y - 1, x)];
        acc = acc + w[2] * a[IDX(y - 1, x + 1)];
        acc = acc + w[3] * a[IDX(y, x - 1)];
        acc = acc + w[4] * a[IDX(y, x)];
        acc = acc + w[5] * a[IDX(y, x + 1)];
        acc = acc + w[6] * a[IDX(y + 1, x - 1)];
        acc = acc + w[7] * a[IDX(y + 1, x)];
        acc = acc + w[8] * a[IDX(y + 1, x + 1)];
        b[IDX(y, x)] = acc;
      }
    }
    for (int x = 0; x < nx + 2; ++x) {
      b[IDX(0, x)] = a[IDX(0, x)];
      b[IDX(ny + 1, x)] = a[IDX(ny + 1, x)];
    }
    for (int yy = 1; yy <= ny; ++yy) {
      b[IDX(yy, 0)] = a[IDX(yy, 0)];
      b[IDX(yy, nx + 1)] = a[IDX(yy, nx + 1)];
    }
    float *tmp = a; a = b; b = tmp;
  }
  memcpy(uT, a, n * sizeof(float));
  free(a);
  free(b);
  (void)nthreads;
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
