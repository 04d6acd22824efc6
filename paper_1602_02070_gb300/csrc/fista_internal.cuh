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

// ---------------------------------------------------------------- tiles --
// A rr x rc matrix is cut into TB x TB tiles. A tile stages the neighbour
// lists of its rows (Lr) and columns (Lc) in shared memory, as element
// offsets into a row-major (ld rc) and a column-major (ld rr) copy of the
// matrix, so that both graph products read contiguous 128-byte segments:
//   (Lr Z)(i, j) = sum_k Lr[i, k] Z(k, j)   -> segments of rows of Z,
//   (Z Lc)(i, j) = sum_k Lc[j, k] ZT(k, i)  -> segments of rows of ZT.
constexpr int TB = 32;        // tile edge
constexpr int kTileNbr = 40;  // neighbour-list entries staged per row / column

template <typename Off>
struct TileNbrT {
  Off roff[TB][kTileNbr];  // element offset of neighbour row k in Z  (k * rc)
  float rval[TB][kTileNbr];
  Off coff[TB][kTileNbr];  // element offset of neighbour row k in ZT (k * rr)
  float cval[TB][kTileNbr];
  int rdeg[TB], cdeg[TB];
  int64_t rf0[TB], cf0[TB];
};
using TileNbr = TileNbrT<int64_t>;
using TileNbr32 = TileNbrT<int32_t>;  // matrices below 2^31 entries

template <typename Off>
__device__ __forceinline__ void stage_nbr(TileNbrT<Off>& nb, const CsrView& Lr, const CsrView& Lc, int rr,
                                          int rc, int i0, int j0, int ni, int nj) {
  if (threadIdx.x < TB) {
    const int r = threadIdx.x;
    const int64_t f0 = r < ni ? Lr.rowptr[i0 + r] : 0;
    nb.rf0[r] = f0;
    nb.rdeg[r] = r < ni ? int(Lr.rowptr[i0 + r + 1] - f0) : 0;
  } else if (threadIdx.x < 2 * TB) {
    const int c = threadIdx.x - TB;
    const int64_t g0 = c < nj ? Lc.rowptr[j0 + c] : 0;
    nb.cf0[c] = g0;
    nb.cdeg[c] = c < nj ? int(Lc.rowptr[j0 + c + 1] - g0) : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * kTileNbr; e += blockDim.x) {
    const int r = e / kTileNbr, q = e % kTileNbr;
    if (q < min(nb.rdeg[r], kTileNbr)) {
      nb.roff[r][q] = Off(int64_t(__ldg(Lr.col + nb.rf0[r] + q)) * rc);
      nb.rval[r][q] = __ldg(Lr.val + nb.rf0[r] + q);
    }
    if (q < min(nb.cdeg[r], kTileNbr)) {
      nb.coff[r][q] = Off(int64_t(__ldg(Lc.col + nb.cf0[r] + q)) * rr);
      nb.cval[r][q] = __ldg(Lc.val + nb.cf0[r] + q);
    }
  }
  __syncthreads();
}

// One staged neighbour list, four consecutive outputs per lane:
// out[t] = sum_q w[q] x[off[q] + base + t], base a multiple of 4 floats
// (16-byte loads from rows whose length is padded to a multiple of 4).
// Entries in list order; beyond the staging area straight from the CSR.
template <typename Off, int CHUNK = 8>
__device__ __forceinline__ float4 nbr_sum_v4(const Off* off, const float* w, int deg, int64_t f0, bool valid,
                                             const float* __restrict__ x, int64_t base, const CsrView& L,
                                             int64_t stride) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!valid) return acc;
  const int ds = min(deg, kTileNbr);
  int q = 0;
  for (; q + CHUNK <= ds; q += CHUNK) {
    float4 v[CHUNK];
#pragma unroll
    for (int t = 0; t < CHUNK; ++t) v[t] = __ldcg(reinterpret_cast<const float4*>(x + off[q + t] + base));
#pragma unroll
    for (int t = 0; t < CHUNK; ++t) {
      const float wt = w[q + t];
      acc.x = fmaf(wt, v[t].x, acc.x);
      acc.y = fmaf(wt, v[t].y, acc.y);
      acc.z = fmaf(wt, v[t].z, acc.z);
      acc.w = fmaf(wt, v[t].w, acc.w);
    }
  }
  for (; q < ds; ++q) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(x + off[q] + base));
    const float wt = w[q];
    acc.x = fmaf(wt, v.x, acc.x);
    acc.y = fmaf(wt, v.y, acc.y);
    acc.z = fmaf(wt, v.z, acc.z);
    acc.w = fmaf(wt, v.w, acc.w);
  }
  for (int64_t f = f0 + kTileNbr; f < f0 + deg; ++f) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(x + int64_t(__ldg(L.col + f)) * stride + base));
    const float wt = __ldg(L.val + f);
    acc.x = fmaf(wt, v.x, acc.x);
    acc.y = fmaf(wt, v.y, acc.y);
    acc.z = fmaf(wt, v.z, acc.z);
    acc.w = fmaf(wt, v.w, acc.w);
  }
  return acc;
}

// Per-instance scratch of a FISTA solve.
struct InstWs {
  float* Z0;          // Z_j ping (row-major)
  float* Z1;          // Z_j pong
  float* ZT0;         // Z_j^T ping (column-major copy)
  float* ZT1;         // Z_j^T pong
  double* scal;       // [|Lr|, |Lc|, lambda, spare]
  double* stats;      // FISTA statistics ring [4][2]
  int* done;          // [stopped, iterations]
};

// Extra scratch of the striped launch of a large single problem: Y~, S and
// one more iterate stripe-major in the processing order, the columns'
// locality order and the ordering kernel's scratch (all null when the
// problem cannot take the striped launch).
struct StripeWs {
  float* Yb;
  float* Sb;
  float* Pb;            // S_{j0-1} in (warm start), S_{J-1} out
  int32_t* perm;        // processing position -> column
  int32_t* inv;         // column -> processing position
  unsigned char* oscr;  // order_scratch_bytes
  unsigned int* bar;    // the ordering kernel's grid barrier
  unsigned int* ctr;    // per-launch stripe counters (a ring of three)
};

// Scratch of a (batched) solve: shared barrier state plus one InstWs each.
struct BatchWs {
  unsigned int* bar;  // grid barrier counter + generation
  int* err;           // barrier timeout flag
  double* part;       // objective partials
  double* obj;
  void* pscr;         // power iteration scratch (power_scratch_bytes)
  InstWs inst[kMaxBatch];
  StripeWs stripe;      // single problems only
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
  // warm start of a single solve: j0 iterations done, X holds S_{j0},
  // warm_prev S_{j0-1}; prev_out (optional) receives S_{J-1} (ld ldx)
  int j0 = 0;
  const float* warm_prev = nullptr;
  float* prev_out = nullptr;
};

// zcols > 0: the Z buffers hold rr x zcols floats (the striped launch's
// stripe-major Z, stripe_zcols(rc)).
InstWs inst_layout(Carve& c, int rr, int rc, size_t zcols = 0);
BatchWs batch_layout(void* ws, const int* rr, const int* rc, int n);
cpca_status fista_batch_run(const BatchProblem* P, int n, int J, double eps, bool want_last,
                            int power_iters, uint64_t power_seed, int blocks, const BatchWs& w,
                            cudaStream_t st, bool dense = false);
// Striped FISTA for single large problems (fista_stripe.cu): one launch per
// iteration, each stripe of Z_j brought into shared memory by a bulk copy;
// the same iterates as the resident and streaming launches. It sets up Z_1
// (or Z_{j0+1}) itself; t0 = t_{j0+1} and mu0 = mu_{j0} of a warm start (1
// and 0 for a cold one); P.prev_out, when set, receives S_{J-1}.
// stripe_candidate: the sizes for which the workspace carries the striped
// launch's scratch (stripe_layout, and Z buffers of stripe_zcols(rc)
// columns); stripe_eligible: the launch is taken (also device limits);
// stripe_reorders: it processes the columns in their locality order.
constexpr int kStripeMaxRows = 5600;
bool stripe_candidate(int rr, int rc);
size_t stripe_zcols(int rc);
bool stripe_eligible(int rr, int rc);
bool stripe_reorders(int rr, int rc);
StripeWs stripe_layout(Carve& c, int rr, int rc);
cpca_status fista_stripe_run(const BatchProblem& P, const InstWs& iw, const StripeWs& sw, int J, double eps,
                             bool want_last, double t0, float mu0, int* err, cudaStream_t st);
// Locality order of a graph's nodes (order.cu): perm[position] = node,
// inv[node] = position; components, then breadth-first levels, then index.
bool order_supported(int n);
size_t order_scratch_bytes(int n);
cpca_status graph_order(const CsrView& L, int32_t* perm, int32_t* inv, void* scratch, unsigned int* bar,
                        int* err, cudaStream_t st);
cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            double* part, double* out, cudaStream_t st);
cpca_status check_csr(const cpca_csr* L, int n, const char* name);

// Power iterations on a few Laplacians with every iterate kept (the solve's
// step size, Sec. IV-B, taken for reverse mode): u_0 = SplitMix64 uniform
// - 1/2 on stream `stream`, u_{t+1} = L u_t / |u_t|, rho = Rayleigh quotient
// of u_T. Forward writes U, nrm2 and *rho; reverse reads them with *rho_bar
// and writes Ub (ubar_t). One thread-block cluster; power_tape_fits says
// whether the rows fit.
struct PowerTape {
  CsrView L;
  int stream;
  float* U;               // [(T + 1) * n]
  double* nrm2;           // [T + 1]
  float* Ub;              // [T * n]
  double* rho;
  const double* rho_bar;
};
bool power_tape_fits(const CsrView* L, int ng);
// Lemma 1 on one graph (decode.cu): S (N x ldo) with S(omega, :) = R and
// (L S)(complement, :) = 0, by Jacobi PCG to tol; workspace
// harmonic_ws_bytes(N, rho, k, nnz of L).
size_t harmonic_ws_bytes(int N, int rho, int k, int64_t nnz);
cpca_status harmonic_extend(const cpca_csr* L, const int32_t* omega, int N, int rho, const float* R, int ldr,
                            int k, double tol, int maxit, float* S, int ldo, int* iters_max, double* res_max,
                            void* ws, cudaStream_t st);
// rho of [0, N) by the sampling generator on SplitMix64 stream `stream`
// (sample.cu), ascending.
cpca_status select_indices(uint64_t seed, int N, int rho, int stream, int32_t* out, cudaStream_t st);

// Scratch of the grid-wide power kernel for graphs of these sizes (the
// one-cluster kernel needs none).
size_t power_scratch_bytes(const int* n, int ng);
// Forward (reverse = false): the one-cluster kernel when the rows fit, else
// the grid-wide kernel with the same arithmetic (scratch: power_scratch_bytes).
// Reverse: one cluster only (returns CPCA_ERR_INVALID_ARG otherwise).
// bar/err: grid-barrier state for the grid-wide kernel (zeroed here).
cpca_status power_tape_run(const PowerTape* P, int ng, int T, uint64_t seed, bool reverse, void* scratch,
                           unsigned int* bar, int* err, cudaStream_t st);
int coop_blocks(const void* kernel, int threads, size_t smem, int want);
// dloss/dL (FP64 on the CSR pattern) -> dloss/dw per entry (adjoint.cu);
// deg and dD are scratch of L.n doubles each.
cpca_status laplacian_weight_grad(const CsrView& L, const float* w, const double* dL, int lap_type,
                                  float* dw, double* deg, double* dD, cudaStream_t st);

}  // namespace cpca
