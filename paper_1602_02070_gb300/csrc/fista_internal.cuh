// fista_internal.cuh - FISTA building blocks shared by the single solve,
// the batched solve and the adjoint.
#pragma once
#include <vector>

#include "common.cuh"

namespace cpca {

struct CsrView {
  int n;
  const int64_t* rowptr;
  const int32_t* col;
  const float* val;
};

// Largest max_iter for which eps > 0 keeps one statistics slot per iteration.
constexpr int kMaxStatIters = 1 << 20;

struct FistaWs {
  float* Z0;      // Z_j ping
  float* Z1;      // Z_j pong
  double* scal;   // [|Lr|, |Lc|, lambda, spare]
  double* vbuf;   // power-iteration vectors
  double* stats;  // per-iteration [|dZ|^2, |Z|^2]
  int* ctl;       // [stopped, iterations]
  double* part;   // objective partials
  double* obj;
  size_t bytes;
};

FistaWs fista_layout(void* ws, int rr, int rc, int max_iter_stats);
cpca_status power_step(const CsrView& Lr, const CsrView& Lc, int iters, uint64_t seed,
                       double gamma_r, double gamma_c, double step_given, const FistaWs& w,
                       cudaStream_t st);
int fista_rows_per_block(int rc);
cpca_status fista_iteration(int R, const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* Zin, float* Zout, float* S,
                            int64_t lds, const double* lam, double gamma_r, double gamma_c,
                            double mu, int iter1, double eps, const double* prev_stats,
                            double* out_stats, int* ctl, cudaStream_t st);
cpca_status fista_init(const float* Yt, int64_t ldy, int rr, int rc, float* Z, float* S,
                       int64_t lds, cudaStream_t st);
cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            const FistaWs& w, cudaStream_t st);
void fista_momentum(int J, double* mu);
cpca_status check_csr(const cpca_csr* L, int n, const char* name);

}  // namespace cpca
