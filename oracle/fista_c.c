/*
 * fista_c.c - plain FP64 C restatement of FISTA for FRPCAG on the sampled
 * matrix (Sec. IV-B, Eq. frpcag_small with phi = l1, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: the same algorithm as oracle.frpcag_fista (the
 * numpy restatement), written out in C so that the full-size parity tests
 * (a 2000 x 10000 sampled matrix, 300 iterations) and the CPU baseline can
 * run it on every host core in reasonable time. It shares nothing with the
 * CUDA library. Every step is the textbook definition: the two graph
 * products are plain CSR sums, no blocking or fusion beyond what Algorithm 1
 * states. Rows are split over OpenMP threads; each output entry is computed
 * by one thread in a fixed order, so the iterates do not depend on the
 * thread count (only the FP64 sums of the stopping test do, in their last
 * bits).
 *
 *   Z_1 = S_0 = Y~, t_1 = 1; for j = 1..J:
 *     G   = 2 (gamma_c Z_j L_c + gamma_r L_r Z_j)
 *     V   = Z_j - lambda G,  R = V - Y~
 *     S_j = Y~ + sgn(R) max(|R| - lambda, 0)
 *     t_{j+1} = (1 + sqrt(1 + 4 t_j^2)) / 2
 *     Z_{j+1} = S_j + ((t_j - 1) / t_{j+1}) (S_j - S_{j-1})
 *     stop when |Z_{j+1} - Z_j|^2 < eps |Z_j|^2 (eps > 0 only)
 * Output: the last S_j (reading of Algorithm 1's undefined output line).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* (Z L)(i, j) = sum_l Z(i, l) L(l, j): row l of L scatters Z(i, l) into
 * the columns it lists. */
static void right_product(int rr, int rc, const double* Z, const int64_t* rowptr, const int32_t* col,
                          const double* val, double* out) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < rr; ++i) {
    const double* z = Z + (size_t)i * rc;
    double* o = out + (size_t)i * rc;
    for (int j = 0; j < rc; ++j) o[j] = 0.0;
    for (int l = 0; l < rc; ++l)
      for (int64_t e = rowptr[l]; e < rowptr[l + 1]; ++e) o[col[e]] += z[l] * val[e];
  }
}

/* (L Z)(i, j) = sum_k L(i, k) Z(k, j). */
static void left_product(int rr, int rc, const double* Z, const int64_t* rowptr, const int32_t* col,
                         const double* val, double* out) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < rr; ++i) {
    double* o = out + (size_t)i * rc;
    for (int j = 0; j < rc; ++j) o[j] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double v = val[e];
      const double* z = Z + (size_t)col[e] * rc;
      for (int j = 0; j < rc; ++j) o[j] += v * z[j];
    }
  }
}

/* Returns 0, or -1 when scratch cannot be allocated. S (rr x rc, row-major)
 * receives the output; *iters the iterations run, *rel the last
 * |Z_{j+1} - Z_j|^2 / |Z_j|^2. threads <= 0: the OpenMP default. */
int oracle_frpcag_fista(int rr, int rc, const double* Yt, const int64_t* lr_ptr, const int32_t* lr_col,
                        const double* lr_val, const int64_t* lc_ptr, const int32_t* lc_col,
                        const double* lc_val, double gamma_r, double gamma_c, double lam, int J,
                        double eps, int threads, double* S, int* iters, double* rel) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  const size_t m = (size_t)rr * rc;
  double* Z = malloc(m * sizeof(double));
  double* Zn = malloc(m * sizeof(double));
  double* Sp = malloc(m * sizeof(double));
  double* A = malloc(m * sizeof(double));
  double* B = malloc(m * sizeof(double));
  if (!Z || !Zn || !Sp || !A || !B) {
    free(Z), free(Zn), free(Sp), free(A), free(B);
    return -1;
  }
  memcpy(Z, Yt, m * sizeof(double));
  memcpy(Sp, Yt, m * sizeof(double));
  memcpy(S, Yt, m * sizeof(double));
  double t = 1.0;
  *iters = 0;
  *rel = NAN;
  for (int j = 1; j <= J; ++j) {
    right_product(rr, rc, Z, lc_ptr, lc_col, lc_val, A);
    left_product(rr, rc, Z, lr_ptr, lr_col, lr_val, B);
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const double mu = (t - 1.0) / tn;
    double dz = 0.0, nz = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : dz, nz)
    for (size_t e = 0; e < m; ++e) {
      const double g = 2.0 * (gamma_c * A[e] + gamma_r * B[e]);
      const double v = Z[e] - lam * g;
      const double r = v - Yt[e];
      const double a = fabs(r) - lam;
      const double sh = a > 0.0 ? a : 0.0;
      const double s = Yt[e] + (r > 0.0 ? sh : (r < 0.0 ? -sh : 0.0));
      const double zn = s + mu * (s - Sp[e]);
      dz += (zn - Z[e]) * (zn - Z[e]);
      nz += Z[e] * Z[e];
      S[e] = s;
      Zn[e] = zn;
    }
    *rel = nz > 0.0 ? dz / nz : 0.0;
    *iters = j;
    if (eps > 0.0 && dz < eps * nz) break;
    /* S_{j-1} <- S_j, Z_j <- Z_{j+1}, t_j <- t_{j+1} */
    memcpy(Sp, S, m * sizeof(double));
    double* tmp = Z;
    Z = Zn;
    Zn = tmp;
    t = tn;
  }
  free(Z), free(Zn), free(Sp), free(A), free(B);
  return 0;
}
