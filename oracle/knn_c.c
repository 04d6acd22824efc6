/*
 * knn_c.c - plain FP64 C restatement of the exact kNN search of Sec. I
 * (graph construction): for every query point i, the K nearest other points
 * by squared Euclidean distance, summed directly as sum_t (y_it - y_jt)^2 in
 * FP64 (never through |a|^2 + |b|^2 - 2ab), the point itself excluded, ties
 * broken by (d^2, j) ascending.
 *
 * TEST INFRASTRUCTURE ONLY: the same definition as oracle.knn_bruteforce
 * (numpy), in C so that the full-size parity tests can search 10^5 points
 * on every host core. Queries are split over OpenMP threads; each query's
 * list is built by one thread (an insertion list of K entries).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* P: N x d row-major FP32 points (the library's and the generator's
 * storage type; each coordinate is converted to FP64 before differencing).
 * queries[nq] (NULL: all N in order). idx/d2: nq x K outputs. */
int oracle_knn(const float* P, int64_t N, int64_t d, int64_t ld, int K, const int64_t* queries,
               int64_t nq, int threads, int64_t* idx, double* d2) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  if (K < 1 || K >= N) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t t = 0; t < nq; ++t) {
    const int64_t i = queries ? queries[t] : t;
    if (i < 0 || i >= N) {
      bad = 1;
      continue;
    }
    int64_t* I = idx + t * K;
    double* D = d2 + t * K;
    int have = 0;
    const float* a = P + i * ld;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      const float* b = P + j * ld;
      double s = 0.0;
      for (int64_t c = 0; c < d; ++c) {
        const double dx = (double)a[c] - (double)b[c];
        s += dx * dx;
      }
      if (have == K && !(s < D[K - 1] || (s == D[K - 1] && j < I[K - 1]))) continue;
      int pos = have < K ? have++ : K - 1;
      while (pos > 0 && (s < D[pos - 1] || (s == D[pos - 1] && j < I[pos - 1]))) {
        D[pos] = D[pos - 1];
        I[pos] = I[pos - 1];
        --pos;
      }
      D[pos] = s;
      I[pos] = j;
    }
  }
  return bad ? -1 : 0;
}
