/*
 * Plain CPU oracle for the 3D 7-point Jacobi iteration that the paper's
 * proxy application runs (Sec. 4.3, "Proxy Application: Jacobi3D": the
 * Jacobi iterative method in a three-dimensional space, a fixed number of
 * iterations, domain split into cuboid blocks that exchange halos with up to
 * six neighbours).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this file.  It
 * shares no code with the CUDA path and never imports it.
 *
 * The oracle is monolithic: it works on ONE padded array holding the whole
 * grid, with no blocks and no halo exchange.  A decomposed run that exchanges
 * halos correctly must reproduce it bit for bit in FP64 (the block split only
 * changes where a neighbour value is read from, never which value it is).
 *
 * Layout: padded array of (nz+2) x (ny+2) x (nx+2) values, x fastest.
 * Interior points have indices 1..n on every axis; indices 0 and n+1 hold the
 * Dirichlet boundary and are never written.
 *
 * Readings of the paper (it prints neither the stencil nor its coefficients):
 *  - Jacobi for the discrete Laplace equation: the new value is the mean of
 *    the six face neighbours, evaluated as
 *        s = ((u[i-1] + u[i+1]) + (u[j-1] + u[j+1])) + (u[k-1] + u[k+1])
 *    then, in FP64, u' = s * c6 with c6 = 1/6 rounded to double, and in FP32
 *    u' = s / 6 rounded once to float.  Multiplying by the float nearest 1/6
 *    would scale every FP32 update by 1 + 2^-25 (that float exceeds 1/6 by a
 *    third of an ulp), a bias that accumulates over the iterations; the
 *    double nearest 1/6 is off by 2^-55 relative, which stays far below the
 *    FP64 rounding noise for any practical iteration count.
 *  - Residual (the paper runs without convergence checks; this is the
 *    convergence test the solver adds): r = s - 6*u at every interior point,
 *    evaluated in FP64 (FP32 states widened exactly), |r| = sqrt(sum r^2)
 *    summed in i, then j order within a z-plane and then over planes in k
 *    order; b is the same expression with every interior value set to 0, and
 *    rel = |r| / |b|.
 * Compile with -ffp-contract=off: no operation may be fused.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PIDX(i, j, k) \
  ((((size_t)(k)) * (size_t)(ny + 2) + (size_t)(j)) * (size_t)(nx + 2) + (size_t)(i))

static const double C6_F64 = 1.0 / 6.0; /* 1/6 rounded to nearest double */

/* The last operation of an update: FP64 multiplies by the double nearest 1/6,
 * FP32 divides by 6 (IEEE division, one rounding). */
#define FINISH_F64(s) ((s) * C6_F64)
#define FINISH_F32(s) ((s) / 6.0f)

/* One Jacobi sweep over every interior point (Sec. 4.3): v <- FINISH(N(u)).
 * v must already hold the boundary values; only interior points are written.
 * z-planes are independent, so the thread count never changes a value. */
#define DEFINE_SWEEP(NAME, T, FINISH)                                           \
  static void NAME(int64_t nx, int64_t ny, int64_t nz, const T* u, T* v) {      \
    _Pragma("omp parallel for schedule(static)")                              \
    for (int64_t k = 1; k <= nz; ++k) {                                         \
      for (int64_t j = 1; j <= ny; ++j) {                                       \
        for (int64_t i = 1; i <= nx; ++i) {                                     \
          T sx = u[PIDX(i - 1, j, k)] + u[PIDX(i + 1, j, k)];                   \
          T sy = u[PIDX(i, j - 1, k)] + u[PIDX(i, j + 1, k)];                   \
          T sz = u[PIDX(i, j, k - 1)] + u[PIDX(i, j, k + 1)];                   \
          T s = (sx + sy) + sz;                                                 \
          v[PIDX(i, j, k)] = FINISH(s);                                         \
        }                                                                       \
      }                                                                         \
    }                                                                           \
  }
DEFINE_SWEEP(sweep_f64, double, FINISH_F64)
DEFINE_SWEEP(sweep_f32, float, FINISH_F32)

/* n_iters Jacobi iterations in place on the padded array u.  Returns 0, or -1
 * when the scratch copy cannot be allocated. */
#define DEFINE_JACOBI(NAME, SWEEP, T)                                           \
  int NAME(int64_t nx, int64_t ny, int64_t nz, T* u, int64_t n_iters) {         \
    size_t n = (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);          \
    T* v = (T*)malloc(n * sizeof(T));                                           \
    if (!v) return -1;                                                          \
    memcpy(v, u, n * sizeof(T)); /* boundary values of the second copy */       \
    T* a = u;                                                                   \
    T* b = v;                                                                   \
    for (int64_t it = 0; it < n_iters; ++it) {                                  \
      SWEEP(nx, ny, nz, a, b);                                                  \
      T* t = a;                                                                 \
      a = b;                                                                    \
      b = t;                                                                    \
    }                                                                           \
    if (a != u) memcpy(u, a, n * sizeof(T));                                    \
    free(v);                                                                    \
    return 0;                                                                   \
  }
DEFINE_JACOBI(oracle_jacobi_f64, sweep_f64, double)
DEFINE_JACOBI(oracle_jacobi_f32, sweep_f32, float)

static int on_boundary(int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny, int64_t nz) {
  return i == 0 || j == 0 || k == 0 || i == nx + 1 || j == ny + 1 || k == nz + 1;
}

/* Residual of the linear system A u = b behind the Jacobi iteration, with
 * A = 6 I - (sum of interior face neighbours) and b = sum of boundary face
 * neighbours.  Outputs |b - A u| and |b| (2-norms over interior points),
 * always in FP64.  Per-plane partial sums are formed in i, j order and added
 * over k in order, so the result does not depend on the thread count.
 * Returns 0, or -1 when scratch cannot be allocated. */
#define DEFINE_RESIDUAL(NAME, T)                                                \
  int NAME(int64_t nx, int64_t ny, int64_t nz, const T* u, double* r_norm,      \
           double* b_norm) {                                                    \
    double* pr = (double*)calloc((size_t)nz + 1, sizeof(double));               \
    double* pb = (double*)calloc((size_t)nz + 1, sizeof(double));               \
    if (!pr || !pb) {                                                           \
      free(pr);                                                                 \
      free(pb);                                                                 \
      return -1;                                                                \
    }                                                                           \
    _Pragma("omp parallel for schedule(static)")                              \
    for (int64_t k = 1; k <= nz; ++k) {                                         \
      double ar = 0.0, ab = 0.0;                                                \
      for (int64_t j = 1; j <= ny; ++j) {                                       \
        for (int64_t i = 1; i <= nx; ++i) {                                     \
          int64_t ni[6] = {i - 1, i + 1, i, i, i, i};                           \
          int64_t nj[6] = {j, j, j - 1, j + 1, j, j};                           \
          int64_t nk[6] = {k, k, k, k, k - 1, k + 1};                           \
          double w[6], wb[6];                                                   \
          for (int q = 0; q < 6; ++q) {                                         \
            w[q] = (double)u[PIDX(ni[q], nj[q], nk[q])];                        \
            wb[q] = on_boundary(ni[q], nj[q], nk[q], nx, ny, nz) ? w[q] : 0.0;  \
          }                                                                     \
          double s = ((w[0] + w[1]) + (w[2] + w[3])) + (w[4] + w[5]);           \
          double sb = ((wb[0] + wb[1]) + (wb[2] + wb[3])) + (wb[4] + wb[5]);    \
          double six_u = 6.0 * (double)u[PIDX(i, j, k)];                        \
          double r = s - six_u;                                                 \
          double r2 = r * r;                                                    \
          double b2 = sb * sb;                                                  \
          ar = ar + r2;                                                         \
          ab = ab + b2;                                                         \
        }                                                                       \
      }                                                                         \
      pr[k] = ar;                                                               \
      pb[k] = ab;                                                               \
    }                                                                           \
    double sr = 0.0, sb = 0.0;                                                  \
    for (int64_t k = 1; k <= nz; ++k) {                                         \
      sr = sr + pr[k];                                                          \
      sb = sb + pb[k];                                                          \
    }                                                                           \
    free(pr);                                                                   \
    free(pb);                                                                   \
    *r_norm = sqrt(sr);                                                         \
    *b_norm = sqrt(sb);                                                         \
    return 0;                                                                   \
  }
DEFINE_RESIDUAL(oracle_residual_f64, double)
DEFINE_RESIDUAL(oracle_residual_f32, float)

/* Solve status codes (shared meaning with the library's, defined here again). */
#define ORACLE_CONVERGED 0
#define ORACLE_MAX_ITERS 1
#define ORACLE_STAGNATED 2

/* Iterate until the relative residual of the current iterate is <= tol.
 * The residual is evaluated on u_k (before the step) whenever k is a multiple
 * of check_every, and at k == max_iters.  Stops with CONVERGED when rel <= tol,
 * MAX_ITERS at the cap, or STAGNATED when `stall_checks` > 0 consecutive
 * checks have not lowered the best relative residual seen.  On return u holds
 * u_k for the reported k.  A zero |b| gives rel = |r| (absolute test).
 * Returns 0, or -1 on allocation failure / bad arguments. */
#define DEFINE_SOLVE(NAME, JACOBI, RESID, T)                                    \
  int NAME(int64_t nx, int64_t ny, int64_t nz, T* u, double tol,                \
           int64_t max_iters, int64_t check_every, int64_t stall_checks,        \
           int64_t* iters_out, double* rel_out, int* status_out) {              \
    if (check_every < 1 || max_iters < 0) return -1;                            \
    double best = INFINITY;                                                     \
    int64_t since = 0;                                                          \
    int64_t k = 0;                                                              \
    for (;;) {                                                                  \
      if (k % check_every == 0 || k == max_iters) {                             \
        double rn, bn;                                                          \
        if (RESID(nx, ny, nz, u, &rn, &bn)) return -1;                          \
        double rel = bn > 0.0 ? rn / bn : rn;                                   \
        *rel_out = rel;                                                         \
        *iters_out = k;                                                         \
        if (rel <= tol) {                                                       \
          *status_out = ORACLE_CONVERGED;                                       \
          return 0;                                                             \
        }                                                                       \
        if (k >= max_iters) {                                                   \
          *status_out = ORACLE_MAX_ITERS;                                       \
          return 0;                                                             \
        }                                                                       \
        if (rel < best) {                                                       \
          best = rel;                                                           \
          since = 0;                                                            \
        } else if (stall_checks > 0 && ++since >= stall_checks) {               \
          *status_out = ORACLE_STAGNATED;                                       \
          return 0;                                                             \
        }                                                                       \
      }                                                                         \
      if (JACOBI(nx, ny, nz, u, 1)) return -1;                                  \
      ++k;                                                                      \
    }                                                                           \
  }
DEFINE_SOLVE(oracle_solve_f64, oracle_jacobi_f64, oracle_residual_f64, double)
DEFINE_SOLVE(oracle_solve_f32, oracle_jacobi_f32, oracle_residual_f32, float)

/* Number of OpenMP threads the sweeps use (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
void oracle_set_threads(int n) { omp_set_num_threads(n); }
#else
int oracle_threads(void) { return 1; }
void oracle_set_threads(int n) { (void)n; }
#endif
