/*
 * Oracle, part 3: unpreconditioned conjugate gradients on an assembled CSR matrix, FP64, OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links or calls this file; only tests/ and the
 * CPU-baseline legs of bench.py load it (through oracle/cg_native.py), to time the oracle's solve of
 * K u = b (Sec. 3.1, Eq. lin_system) on all host cores and on one.
 *
 * The iteration is the textbook CG recurrence written out once, in the same order as
 * oracle/solvers.py::cg (which the tests hold it to):
 *     r = b - K x,  p = r,  rr = <r, r>
 *     repeat while sqrt(rr / <b, b>) > tol:  Kp = K p;  alpha = rr / <p, Kp>;  x += alpha p;
 *                                            r -= alpha Kp;  rr' = <r, r>;  p = r + (rr' / rr) p
 * The matrix-vector product is a plain CSR row loop; rows and dot products are split over OpenMP
 * threads with static schedules (the dot products' rounding therefore depends on the thread count,
 * which only affects the last bits).  No preconditioner, no blocking, no reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t* indptr, const int32_t* indices, const double* data, const double* x,
                 double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t k = indptr[i]; k < indptr[i + 1]; ++k) acc += data[k] * x[indices[k]];
    y[i] = acc;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Solves K x = b from the x passed in (x is overwritten with the iterate).  Returns the number of
 * iterations taken, or -1 when the scratch cannot be allocated; *relres receives sqrt(<r, r> / <b, b>).
 * nthreads > 0 fixes the OpenMP thread count of this call.  Stops after maxiter iterations, or when the
 * residual norm has not halved for 2000 iterations (stagnation), as the Python version does. */
int csr_cg(int64_t n, const int64_t* indptr, const int32_t* indices, const double* data, const double* b,
           double* x, double tol, int maxiter, int nthreads, double* relres) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* Kp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !Kp) {
    free(r);
    free(p);
    free(Kp);
    return -1;
  }
  spmv(n, indptr, indices, data, x, Kp);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - Kp[i];
    p[i] = r[i];
  }
  double rr = dot(n, r, r);
  const double bb = dot(n, b, b);
  int it = 0;
  if (bb == 0.0) {
    *relres = 0.0;
    free(r);
    free(p);
    free(Kp);
    return 0;
  }
  double best = INFINITY;
  int stall = 0;
  while (it < maxiter) {
    if (sqrt(rr / bb) <= tol) break;
    spmv(n, indptr, indices, data, p, Kp);
    const double alpha = rr / dot(n, p, Kp);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Kp[i];
    }
    const double rr_new = dot(n, r, r);
    const double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    ++it;
    const double rel = sqrt(rr / bb);
    if (rel < 0.5 * best) {
      best = rel;
      stall = 0;
    } else if (++stall > 2000) {
      break;
    }
  }
  *relres = sqrt(rr / bb);
  free(r);
  free(p);
  free(Kp);
  return it;
}

/* Number of threads an OpenMP parallel region of this library would use by default (1 without OpenMP). */
int csr_cg_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
