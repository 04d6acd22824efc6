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

// Kept for the workspace-size signature (statistics now live in a ring).
constexpr int kMaxStatIters = 1 << 20;
constexpr int kObjBlocks = 512;

struct FistaWs {
  float* Z0;          // Z_j ping
  float* Z1;          // Z_j pong
  float* ZT0;         // Z_j^T ping (column-major copy)
  float* ZT1;         // Z_j^T pong
  double* scal;       // [|Lr|, |Lc|, lambda, spare]
  float* pu[2][2];    // power iteration vectors [graph][ping/pong]
  double* pacc;       // power iteration norm ring [3][2] + quotients [2][2]
  double* stats;      // FISTA statistics ring [4][2]
  int* ctl;           // [stopped, iterations]
  unsigned int* bar;  // grid barrier counters + generation
  int* err;           // barrier timeout flag
  double* part;       // objective partials
  double* obj;
  size_t bytes;
};

FistaWs fista_layout(void* ws, int rr, int rc, int unused);
cpca_status power_step(const CsrView& Lr, const CsrView& Lc, int iters, uint64_t seed,
                       double gamma_r, double gamma_c, double step_given, const FistaWs& w,
                       cudaStream_t st);
cpca_status fista_run(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                      const CsrView& Lc, float* X, int64_t ldx, double gamma_r, double gamma_c,
                      int J, double eps, bool want_last, int tile_rows, const FistaWs& w,
                      cudaStream_t st);
cpca_status fista_init(const float* Yt, int64_t ldy, int rr, int rc, float* Z, float* ZT,
                       float* S, int64_t lds, cudaStream_t st);
cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            const FistaWs& w, cudaStream_t st);
void fista_momentum(int J, double* mu);
cpca_status check_csr(const cpca_csr* L, int n, const char* name);

}  // namespace cpca
