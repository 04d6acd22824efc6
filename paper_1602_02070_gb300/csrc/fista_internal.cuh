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

constexpr int kMaxBatch = 128;  // instances per batched call (kernel-parameter table)
constexpr int kObjBlocks = 512;

// Per-instance scratch of a FISTA solve.
struct InstWs {
  float* Z0;          // Z_j ping (row-major)
  float* Z1;          // Z_j pong
  float* ZT0;         // Z_j^T ping (column-major copy)
  float* ZT1;         // Z_j^T pong
  double* scal;       // [|Lr|, |Lc|, lambda, spare]
  float* pu[2][2];    // power iteration vectors [graph][ping/pong]
  double* pacc;       // power iteration norm rings [2][3] + quotients [2][2]
  double* stats;      // FISTA statistics ring [4][2]
  int* done;          // [stopped, iterations]
};

// Scratch of a (batched) solve: shared barrier state plus one InstWs each.
struct BatchWs {
  unsigned int* bar;  // grid barrier counter + generation
  int* err;           // barrier timeout flag
  double* part;       // objective partials
  double* obj;
  InstWs inst[kMaxBatch];
  int n;
  size_t bytes;
};

struct BatchProblem {
  const float* Yt;
  int64_t ldy;
  int rr, rc;
  CsrView Lr, Lc;
  double gamma_r, gamma_c, step;
  float* X;
  int64_t ldx;
};

InstWs inst_layout(Carve& c, int rr, int rc);
BatchWs batch_layout(void* ws, const int* rr, const int* rc, int n);
cpca_status fista_batch_run(const BatchProblem* P, int n, int J, double eps, bool want_last,
                            int power_iters, uint64_t power_seed, int blocks, const BatchWs& w,
                            cudaStream_t st);
cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            double* part, double* out, cudaStream_t st);
cpca_status check_csr(const cpca_csr* L, int n, const char* name);
int coop_blocks(const void* kernel, int threads, size_t smem, int want);

}  // namespace cpca
