/*
 * cpca.h - C ABI of the GB300 compressive-PCA-on-graphs library (libcpca.so).
 *
 * The library implements the data-parallel hot path of compressive PCA on
 * graphs (Shahid, Perraudin, Puy, Vandergheynst, arXiv 1602.02070):
 *   - kNN graphs and Laplacians between rows or columns   (Sec. I, Sec. VII-A)
 *   - uniform row/column sampling, Y~ = M_r Y M_c         (Sec. III, Eq. Mc)
 *   - FRPCAG on the sampled matrix by FISTA               (Sec. IV-B, Algorithm 1)
 *   - the subspace-upsampling approximate decoder         (Sec. V-C, Lemma 1,
 *                                                          Eq. Uupsample, Algorithm 2)
 *   - the alternate, clustering and projection decoders   (Sec. V-B, Algorithm 3,
 *                                                          appendix)
 *   - Kron-reduced compressed Laplacians                  (Sec. IV-A)
 *   - reverse-mode derivatives and batched solves         (not in the paper)
 *
 * Conventions (all entry points):
 *   - Array arguments are DEVICE pointers unless marked "host". The caller
 *     owns and allocates every buffer; the library allocates no device
 *     memory of its own. Calls that need scratch take (ws, ws_bytes) and
 *     have a *_workspace_size query; ws must be 256-byte aligned.
 *   - Matrices are FP32, row-major, with an explicit leading dimension
 *     (elements between consecutive rows, >= the row length).
 *   - Indices are int32 (sizes < 2^31); CSR row pointers are int64.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless it says it synchronises.
 *   - Every call returns a cpca_status; on failure cpca_last_error() gives
 *     a message (thread-local). No C++ exception crosses the ABI. Argument
 *     errors are detected on the host before anything is launched.
 *   - Kernels never wait without bound: every device-side wait has an
 *     iteration limit and reports CPCA_ERR_TIMEOUT instead of hanging.
 */
#ifndef CPCA_H
#define CPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cpca_status;
#define CPCA_OK                0
#define CPCA_ERR_INVALID_ARG   1  /* bad size, pointer, alignment or parameter */
#define CPCA_ERR_CUDA          2  /* a CUDA runtime call or kernel launch failed */
#define CPCA_ERR_WORKSPACE     3  /* ws_bytes smaller than the *_workspace_size query */
#define CPCA_ERR_SINGULAR      4  /* L_aa not invertible (a component has no sampled node) */
#define CPCA_ERR_NOT_CONVERGED 5  /* iteration cap reached before the tolerance */
#define CPCA_ERR_TIMEOUT       6  /* a bounded device-side wait gave up */
#define CPCA_ERR_CAPACITY      7  /* an output buffer is too small (e.g. nnz_cap) */
#define CPCA_ERR_NONFINITE     8  /* NaN or Inf in a result that reports its objective */

#define CPCA_LAP_NORMALIZED    0  /* L_n = D^-1/2 (D - W) D^-1/2 (Sec. I) */
#define CPCA_LAP_COMBINATORIAL 1  /* L = D - W (Sec. I) */

/* Message of the last failed call on this host thread ("" if none). */
const char* cpca_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int32_t cpca_version(void);
/* Number of kernels this library has launched in this process. */
uint64_t cpca_launch_count(void);

/* Failure-path hooks (not in the paper; for tests of the error paths
 * without a GPU fault).
 * cpca_debug_set_barrier_spin_limit(polls): grid-barrier waits of launches
 * made after this call give up after `polls` polls (polls <= 0 restores the
 * default, about a second of waiting); a wait that gives up sets the
 * launch's error flag, every block leaves its loops and the call reports
 * CPCA_ERR_TIMEOUT. Process-wide; returns 0.
 * Environment variable CPCA_FAULT (read at every call): "timeout" acts as a
 * poll limit of 1; "nan" makes cpca_frpcag_solve write a NaN into X[0][0]
 * after the solve (so a call with `info` reports CPCA_ERR_NONFINITE); the
 * Python binding also takes "alloc" (its workspace allocation fails before
 * any launch). */
int32_t cpca_debug_set_barrier_spin_limit(int64_t polls);

/* Per-kernel CUDA-event timing (tracing aid; off by default).
 * cpca_profile_enable(on, prefix) clears earlier records and, when on != 0,
 * brackets every later launch whose kernel name starts with `prefix`
 * (NULL or "" = all named kernels) with a pair of CUDA events on the launch
 * stream. cpca_profile_read() waits for those events and writes, per kernel
 * name (up to max_names, names in a max_names x name_len host char array),
 * the summed milliseconds and the launch count; it returns the number of
 * distinct names recorded. Kernel names: knn_candidates_tc,
 * knn_candidates_simt, knn_recheck, fista_iter, cg_pcg, decode_output, ... */
int32_t cpca_profile_enable(int32_t on, const char* name_prefix);
int32_t cpca_profile_read(int32_t max_names, char* names, int32_t name_len, double* total_ms,
                          int32_t* launches);

/* Sparse symmetric Laplacian in CSR form: n x n, nnz stored entries,
 * column indices ascending within each row, the diagonal stored explicitly.
 * rowptr[n+1] int64, col[nnz] int32, val[nnz] FP32; all device pointers. */
typedef struct cpca_csr {
  int32_t n;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const float* val;
} cpca_csr;

/* ------------------------------------------------------------------------
 * cpca_knn_graph - exact kNN graph and its Laplacian (Sec. I; Sec. VII-A).
 *
 * Points: if transposed == 0, point i is row i of `pts` (npts rows of `dim`
 * floats, leading dimension ld >= dim); if transposed == 1, point i is
 * column i of a dim x npts row-major matrix with leading dimension ld >= npts
 * (pass Y with npts = n, dim = p, ld = n for the column graph of Y).
 * For each point the K nearest other points by Euclidean distance are found
 * (ties by lower index). Candidates are ranked by |a|^2 + |b|^2 - 2ab with the
 * dot products on the tensor cores (a copy of the points scaled by a power
 * of two and rounded to half precision - the significand of TF32 - with
 * FP32 accumulation; FP32 SIMT on other GPUs); the kept squared distances are then
 * summed directly over the coordinates in FP32, and a certificate (the
 * ranking error bound against the gap to the best non-candidate) decides
 * per query whether an exact brute-force search is needed. The graph joins i and j if either is among the other's
 * K nearest; W_ij = exp(-d2_ij / sigma2) with sigma2 = the given value, or,
 * if sigma2 <= 0, the mean of the npts*K directed kNN squared distances.
 * Degrees D_ii = sum_j W_ij; lap_type selects L_n (CPCA_LAP_NORMALIZED) or
 * L = D - W (CPCA_LAP_COMBINATORIAL); a node with zero degree gets an
 * all-zero row in L_n.
 *
 * Outputs (device): CSR rowptr[npts+1], col[nnz], val[nnz] (the Laplacian,
 * diagonal included), weight[nnz] (W_ij on the same pattern, 0 on the
 * diagonal; may be NULL); knn_idx[npts*K], knn_d2[npts*K] (may be NULL).
 * nnz_cap must be >= npts*(2K+1) (the largest possible pattern).
 * Host outputs: *nnz_out, *sigma2_out (either may be NULL).
 * Workspace: cpca_knn_graph_workspace_size (it includes the half copy,
 * 2 npts dim bytes).
 * This call SYNCHRONISES `stream` once (to return nnz).
 * Requirements: 1 <= K <= 32, K < npts, dim >= 1.
 * ---------------------------------------------------------------------- */
size_t cpca_knn_graph_workspace_size(int32_t npts, int32_t dim, int32_t K, int32_t transposed);
/* Certification record of the last cpca_knn_graph call on this host
 * thread. The tensor-core candidates of a query are certified when the
 * worst-case error bound of the half-precision ranking proves that no point outside its candidate
 * lists can beat the K-th exact distance. Queries that fail are searched
 * by exact brute force while their number stays within a budget of
 * max(64, 2e11 / (npts dim)) (a query costs npts dim FMAs):
 * cpca_knn_last_bruteforce() counts them. Beyond the budget none is
 * redone; each keeps the exact K nearest of the 2K best of its tensor-core
 * candidates (the ranking error is far below the distance gaps in
 * practice, but the worst-case bound can exceed the spread of a tight
 * cluster in high dimension) and cpca_knn_last_uncertified() counts them.
 * cpca_knn_last_err_rel() is the relative part of that bound (times
 * |q|^2 + |b|^2) for the same call: 2^-10 + 2^-22 + (t + 8 + c) 2^-23 for
 * the tensor-core ranking, t the products in one tensor-core accumulation
 * (dim up to 32768 dimensions, one accumulation; above, 4096 per
 * accumulation chunk) and c the chunks (0 when unchunked); the FP32 SIMT
 * ranking's bound otherwise. */
int32_t cpca_knn_last_bruteforce(void);
int32_t cpca_knn_last_uncertified(void);
double cpca_knn_last_err_rel(void);
cpca_status cpca_knn_graph(const float* pts, int32_t npts, int32_t dim, int64_t ld,
                           int32_t transposed, int32_t K, int32_t lap_type, double sigma2,
                           int64_t* rowptr, int32_t* col, float* val, float* weight,
                           int64_t nnz_cap, int32_t* knn_idx, float* knn_d2,
                           int64_t* nnz_out, double* sigma2_out,
                           void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * cpca_sample - uniform sampling without replacement (Sec. III, Eq. Mc).
 *
 * Draws Omega_r (rho_r of [0,p)) and Omega_c (rho_c of [0,n)), each in
 * ascending order, and gathers Yt = Y(Omega_r, Omega_c) = M_r Y M_c, a
 * rho_r x rho_c matrix (leading dimension ldyt). Index i of side s
 * (s = 0 rows, 1 columns) gets the key k_i = SplitMix64 output i+1 of the
 * generator whose state starts at seed XOR (0x9E3779B97F4A7C15 * (s+1));
 * Omega is the rho indices with the smallest (k_i, i). Y and Yt may both be
 * NULL to draw only the indices. No workspace.
 * Requirements: 0 < rho_r <= p, 0 < rho_c <= n.
 * ---------------------------------------------------------------------- */
cpca_status cpca_sample(uint64_t seed, int32_t p, int32_t n, int32_t rho_r, int32_t rho_c,
                        const float* Y, int64_t ldy, int32_t* omega_r, int32_t* omega_c,
                        float* Yt, int64_t ldyt, void* stream);

/* ------------------------------------------------------------------------
 * cpca_frpcag_solve - FRPCAG on the sampled matrix by FISTA
 * (Sec. IV-B, Eq. frpcag_small with phi = l1; Algorithm 1).
 *
 *   min_X |Yt - X|_1 + gamma_c tr(X Lc X^T) + gamma_r tr(X^T Lr X)
 *
 * Z_1 = S_0 = Yt, t_1 = 1; per iteration j:
 *   S_j = Yt + sgn(V - Yt) max(|V - Yt| - lambda, 0),
 *         V = Z_j - lambda * 2 (gamma_c Z_j Lc + gamma_r Lr Z_j),
 *   t_{j+1} = (1 + sqrt(1 + 4 t_j^2)) / 2,
 *   Z_{j+1} = S_j + ((t_j - 1) / t_{j+1}) (S_j - S_{j-1}).
 * lambda = params.step if > 0, else 1 / (2 gamma_c |Lc|_2 + 2 gamma_r |Lr|_2)
 * with the norms from `power_iters` power iterations in FP64 (start vector
 * u_i - 1/2, u the SplitMix64 uniforms of (power_seed, stream 2 for Lr,
 * 3 for Lc)), or 1 when that denominator is 0. With eps > 0 the loop stops
 * once |Z_{j+1} - Z_j|_F^2 < eps |Z_j|_F^2 (tested on the device after every
 * iteration); eps = 0 runs exactly max_iter iterations. All iterations run
 * in one cooperative kernel (one bounded grid barrier per iteration), or,
 * for a single problem too large to keep every tile resident, in one striped
 * launch per iteration (see params.blocks; the same iterates bit for bit);
 * the call does not synchronise unless `info` is given. The output X (rr x rc,
 * leading dimension ldx) is the last S_j. FP32 arithmetic, FP64 reductions.
 * Lr is rr x rr, Lc is rc x rc, both symmetric.
 * Dense Laplacians (the Kron reductions of Sec. IV-A): when both CSRs hold
 * n^2 entries, eps = 0 and blocks = 0, the call checks on the device (one
 * synchronisation) that every entry is stored in row-major order, as
 * cpca_kron_reduce returns them; if so, each iteration is one launch of a
 * tiled FP32 contraction of both products with the update fused (no grid
 * barrier), which agrees with the gather kernel to FP32 rounding.
 * `info` (host, may be NULL): if given, the call SYNCHRONISES and fills it,
 * including the FP64 objective of X, and reports CPCA_ERR_TIMEOUT (a grid
 * barrier gave up) or CPCA_ERR_NONFINITE (the objective is NaN or Inf).
 * Without `info` the call is asynchronous and reports neither: the barrier
 * flag stays in `ws` for cpca_frpcag_status.
 * Dense inputs take one synchronisation for the pattern check, so a call on
 * dense Laplacians cannot be captured in a CUDA graph.
 * ---------------------------------------------------------------------- */
typedef struct cpca_frpcag_params {
  double gamma_r;
  double gamma_c;
  double step;          /* lambda; <= 0 selects 1/beta' by power iteration */
  int32_t max_iter;     /* J >= 0 */
  double eps;           /* stopping tolerance; 0 = exactly max_iter iterations */
  int32_t power_iters;  /* power iterations per Laplacian (>= 1) */
  uint64_t power_seed;
  int32_t blocks;       /* FISTA launch width (blocks); 0 = automatic: one block per
                           32 x 32 tile when all tiles fit on the GPU at once;
                           else, for a single problem with 256 <= rr and a
                           stripe of Z in shared memory (rr <= about 2800),
                           the striped launch (one per iteration); else the
                           autotuner's choice for this tile count if
                           cpca_frpcag_tune_batched has run, else the widest
                           co-resident grid. > 0 forces the cooperative
                           kernel with that many blocks. */
  /* Checkpoint and resume of Algorithm 1 (single solves; 0 / NULL for a
   * cold start, and for the batched, tape and backward calls):
   * start_iter = j0 > 0 resumes after iteration j0: on entry X holds S_{j0}
   * and start_prev (device, rr x rc, leading dimension ldx) holds S_{j0-1}
   * (Y~ when j0 = 1); the call computes Z_{j0+1} = S_{j0} + mu_{j0}
   * (S_{j0} - S_{j0-1}) and runs iterations j0+1 .. j0+max_iter, t_j
   * continuing the recurrence. prev_out (device, rr x rc, leading dimension
   * ldx, may be NULL; needs eps = 0) receives S_{J-1}, the iterate before the
   * returned one, so (X, prev_out, j0 + max_iter) resumes the solve. With
   * the same lambda (a given step, or the same power iterations), J1
   * iterations and a resumed J2 give X bit for bit equal to one call of
   * J1 + J2 iterations. */
  int32_t start_iter;
  const float* start_prev;
  float* prev_out;
} cpca_frpcag_params;

typedef struct cpca_solve_info {
  int32_t iters;        /* iterations run */
  double step;          /* lambda used */
  double norm_r;        /* |Lr|_2 estimate (0 if step was given) */
  double norm_c;        /* |Lc|_2 estimate (0 if step was given) */
  double rel_change;    /* |Z_{j+1} - Z_j|^2 / |Z_j|^2 of the last iteration */
  double objective;     /* F(X) in FP64 */
} cpca_solve_info;

size_t cpca_frpcag_workspace_size(int32_t rr, int32_t rc);

/* ------------------------------------------------------------------------
 * Batched FRPCAG: up to 128 independent problems (each its own Y~, sizes,
 * graphs, gammas and optional step) solved by FISTA in ONE cooperative
 * launch (plus one launch for all power iterations): every problem runs the
 * same max_iter iterations of Algorithm 1, or stops on its own when
 * eps > 0. Results equal per-problem cpca_frpcag_solve calls (bit for bit;
 * for dense Laplacians, where the single solve takes its dense kernel, to
 * FP32 rounding). Without
 * `infos` the call is fully asynchronous and may be captured in a CUDA
 * graph (run it once outside capture first). params.gamma_* and .step are
 * ignored (taken from each problem); .max_iter, .eps, .power_iters,
 * .power_seed and .blocks apply to all. `infos` (host, count entries) may
 * be NULL; if given, the call synchronises and fills them.
 * ---------------------------------------------------------------------- */
typedef struct cpca_problem {
  const float* Yt;
  int32_t rr, rc;
  int64_t ldyt;
  cpca_csr Lr, Lc;
  double gamma_r, gamma_c;
  double step;          /* <= 0: 1/beta' by power iteration */
  float* X;
  int64_t ldx;
} cpca_problem;

size_t cpca_frpcag_batched_workspace_size(const cpca_problem* probs, int32_t count);
cpca_status cpca_frpcag_solve_batched(const cpca_problem* probs, int32_t count,
                                      const cpca_frpcag_params* params, cpca_solve_info* infos,
                                      void* ws, size_t ws_bytes, void* stream);
/* Autotuner: times 10-iteration runs of the batched FISTA kernel at each
 * candidate launch width (multiples of the SM count, and one block per tile
 * when that fits) and returns the fastest in *blocks (also remembered for
 * later automatic launches with the same tile count). Synchronises. The
 * problems' X buffers are overwritten. */
cpca_status cpca_frpcag_tune_batched(const cpca_problem* probs, int32_t count, int32_t* blocks,
                                     float* ms_per_10_iters, void* ws, size_t ws_bytes,
                                     void* stream);

cpca_status cpca_frpcag_solve(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                              const cpca_csr* Lr, const cpca_csr* Lc,
                              const cpca_frpcag_params* params,
                              float* X, int64_t ldx, cpca_solve_info* info,
                              void* ws, size_t ws_bytes, void* stream);

/* Status of the last FISTA solve (single, batched or no-allocation) on the
 * workspace `ws` (NULL: the no-allocation solve's built-in scratch):
 * SYNCHRONISES `stream`, then returns CPCA_ERR_TIMEOUT if a grid barrier of
 * that solve's power iterations or FISTA launch gave up, else CPCA_OK.
 * Solves without `info` are asynchronous and never read that flag
 * themselves; call this (after they finish, e.g. after any synchronising
 * call) to learn of a timeout. */
cpca_status cpca_frpcag_status(const void* ws, void* stream);

/* ------------------------------------------------------------------------
 * cpca_frpcag_solve_noalloc - cpca_frpcag_solve without a workspace.
 *
 * (No counterpart in the paper: a deployment convenience.) For callers that
 * cannot allocate device memory: a plugin inside a host application whose
 * memory pool owns the whole device, code that must not call cudaMalloc or
 * cudaFree because they can synchronise the device, or a fixed-budget
 * process that reserves all memory up front. Same arguments, semantics and
 * results as cpca_frpcag_solve, minus (ws, ws_bytes): the scratch is a
 * CPCA_NOALLOC_WS_BYTES array in the library's own device memory (every GPU
 * that loads libcpca.so holds it until the process exits). Problems needing
 * more scratch than that (cpca_frpcag_workspace_size(rr, rc) >
 * CPCA_NOALLOC_WS_BYTES, about rr * rc <= 2 million entries) are rejected
 * with CPCA_ERR_WORKSPACE. Nothing is allocated: no cudaMalloc, cudaFree or
 * allocating library call. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. All calls share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race;
 * each call clears what must start at zero itself.
 * ---------------------------------------------------------------------- */
#define CPCA_NOALLOC_WS_BYTES (32u << 20)
cpca_status cpca_frpcag_solve_noalloc(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                      const cpca_csr* Lr, const cpca_csr* Lc,
                                      const cpca_frpcag_params* params, float* X, int64_t ldx,
                                      cpca_solve_info* info, void* stream);

/* ------------------------------------------------------------------------
 * cpca_frpcag_backward - reverse-mode derivative of cpca_frpcag_solve.
 *
 * (The paper has no derivatives; this differentiates the computed map.)
 * For a loss of the FISTA output X = S_J (Algorithm 1 with a fixed
 * iteration count J = params->max_iter; params->eps must be 0), given
 * dX = dloss/dX, returns the derivatives with respect to
 *   - Y~ (dYt, rr x rc, leading dimension lddyt, FP32, overwritten);
 *   - gamma_r, gamma_c (ginfo), including their effect through
 *     lambda = 1/beta' (Sec. IV-B) when lambda is computed (params->step
 *     <= 0); with a given step, lambda is a constant and ginfo->dlambda
 *     reports dloss/dlambda;
 *   - the values of Lr and Lc on their CSR patterns (dLr, dLc: nnz FP64
 *     each, device, optional), through FISTA and through the power
 *     iterations that estimate |Lr|_2, |Lc|_2 (same start vectors and
 *     count as the solve: the derivative is that of the estimate);
 *   - the edge weights (dwr, dwc: nnz FP32 each, device, optional), given
 *     the weights wr, wc on the same patterns (the `weight` output of
 *     cpca_knn_graph) and lap_type: an undirected edge's derivative is
 *     written at both of its entries, 0 on the diagonal. The Laplacian is
 *     the function of the weights of Sec. I (normalised: the entry and both
 *     degrees move).
 * The prox is differentiated where it is smooth: its derivative is 1 where
 * |Z_j - lambda grad g(Z_j) - Y~| > lambda, else 0.
 * Checkpointing: (S_j, Z_{j+1}) is stored every ckpt_every iterations
 * (0 selects 20; >= max_iter stores the whole trajectory, no recompute);
 * each segment is recomputed once before its reverse sweep. Cost: about
 * two forward solves plus the reverse sweep (two graph products per
 * iteration); scratch from cpca_frpcag_backward_workspace_size.
 * resume != 0: `ws` holds the tape of a cpca_frpcag_forward_tape call with
 * the same inputs, params and ckpt_every (power iterates, lambda and the
 * checkpoints), so the first forward pass is skipped.
 * All device pointers; ginfo is host. SYNCHRONISES the stream.
 *
 * cpca_frpcag_forward_tape: the forward solve (X = S_J, as
 * cpca_frpcag_solve with eps = 0, same arithmetic per entry) that also
 * records the tape in `ws` (cpca_frpcag_backward_workspace_size bytes) for a
 * later cpca_frpcag_backward(..., resume = 1, ...). ginfo (host, optional)
 * receives lambda and the norm estimates. SYNCHRONISES.
 * ---------------------------------------------------------------------- */
typedef struct cpca_frpcag_grad_info {
  double dgamma_r, dgamma_c;  /* total derivatives */
  double dlambda;             /* dloss/dlambda */
  double dnorm_r, dnorm_c;    /* dloss/d|Lr|_2, dloss/d|Lc|_2 (estimates) */
  double lambda;              /* the step used */
  double norm_r, norm_c;      /* the norm estimates (0 if step was given) */
} cpca_frpcag_grad_info;

size_t cpca_frpcag_backward_workspace_size(int32_t rr, int32_t rc, int32_t max_iter,
                                           int32_t ckpt_every, int32_t power_iters,
                                           int64_t nnz_r, int64_t nnz_c);
cpca_status cpca_frpcag_forward_tape(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                     const cpca_csr* Lr, const cpca_csr* Lc,
                                     const cpca_frpcag_params* params, int32_t ckpt_every, float* X,
                                     int64_t ldx, cpca_frpcag_grad_info* ginfo, void* ws,
                                     size_t ws_bytes, void* stream);
cpca_status cpca_frpcag_backward(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                 const cpca_csr* Lr, const cpca_csr* Lc,
                                 const cpca_frpcag_params* params, int32_t ckpt_every,
                                 int32_t resume,
                                 const float* dX, int64_t lddx, float* dYt, int64_t lddyt,
                                 double* dLr, double* dLc, const float* wr, const float* wc,
                                 int32_t lap_type, float* dwr, float* dwc,
                                 cpca_frpcag_grad_info* ginfo, void* ws, size_t ws_bytes,
                                 void* stream);

/* ------------------------------------------------------------------------
 * cpca_decode - subspace-upsampling approximate decoder
 * (Sec. V-C; Lemma 1; Eq. Uupsample; Algorithm 2).
 *
 * 1. Top singular triplets of Xt (rr x rc) by block subspace iteration
 *    with block size b = min(rr, rc, kmax + 8), FP32 products, FP64 Gram /
 *    Cholesky-QR / Jacobi eigen-solve.
 * 2. k = number of singular values with s_i / s_1 >= rank_ratio (or
 *    k_override if > 0); k <= kmax, else CPCA_ERR_INVALID_ARG.
 * 3. For every column, U(Omega_r,:) = U~ and U(a,:) = -Lr_aa^-1 Lr_ab U~
 *    (a = rows not in Omega_r), likewise V on Lc; solved by Jacobi-PCG
 *    (all 2k columns in one cooperative kernel, FP32 vectors, FP64 dots),
 *    per column to |r| <= cg_tol |b| or cg_max_iter iterations.
 * 4. Unit-normalise the columns of U and V.
 * 5. sigma_i = sqrt(n p / (rr rc (1 - delta))) s_i.
 * 6. X = U diag(sigma) V^T (p x n, leading dimension ldx) if X != NULL.
 *    X may be device memory or page-locked host memory that the GPU can
 *    address (cudaHostAlloc, or cudaHostRegister with the mapped flag, on a
 *    system with unified addressing): the output kernel then writes X
 *    straight into host memory over the CPU-GPU link, with no device copy
 *    of the p x n result (the whole 8 GB output of a 20000 x 100000 matrix
 *    never touches HBM).
 *
 * omega_r (rr ascending indices of [0,p)) and omega_c (rc of [0,n)) are the
 * sampling sets of cpca_sample; Lr (p x p) and Lc (n x n) the full graphs.
 * Optional outputs (may be NULL): U (p x kmax, row-major, ld kmax),
 * V (n x kmax, ld kmax), sigma (kmax doubles), all device.
 * Host outputs: *k_out, and `info` if not NULL.
 * This call SYNCHRONISES `stream` (k is needed on the host).
 * Returns CPCA_ERR_NOT_CONVERGED if a column hit cg_max_iter (X is still
 * written), CPCA_ERR_TIMEOUT if a device barrier gave up.
 * ---------------------------------------------------------------------- */
typedef struct cpca_decode_params {
  double rank_ratio;    /* 0.1 in Algorithm 2 */
  int32_t k_override;   /* > 0: use this k */
  int32_t kmax;         /* largest k supported by the buffers (<= 48) */
  double delta;         /* RIP constant in step 5, in [0, 1) */
  double cg_tol;        /* relative residual tolerance */
  int32_t cg_max_iter;  /* <= 0: 10 * (number of unsampled nodes) */
  int32_t svd_iters;    /* subspace iterations (>= 1) */
  uint64_t svd_seed;    /* start block: SplitMix64 uniforms - 1/2, stream 4 */
} cpca_decode_params;

typedef struct cpca_decode_info {
  int32_t k;
  int32_t cg_iters_u;   /* largest iteration count over the U columns */
  int32_t cg_iters_v;   /* same for V */
  double cg_res_u;      /* largest final relative residual over U columns */
  double cg_res_v;
  double s_tilde[64];   /* leading singular values of Xt (first b entries valid) */
  int32_t b;            /* subspace block size used */
} cpca_decode_info;

size_t cpca_decode_workspace_size(int32_t p, int32_t n, int32_t rr, int32_t rc, int32_t kmax,
                                  int64_t nnz_r, int64_t nnz_c);  /* nnz of Lr and Lc */
cpca_status cpca_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                        const int32_t* omega_r, const int32_t* omega_c,
                        int32_t p, int32_t n, const cpca_csr* Lr, const cpca_csr* Lc,
                        const cpca_decode_params* params,
                        float* X, int64_t ldx, float* U, float* V, double* sigma,
                        int32_t* k_out, cpca_decode_info* info,
                        void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * cpca_decode_backward - reverse-mode derivative of cpca_decode.
 *
 * (The paper has no derivatives; this differentiates the computed map with
 * the rank k fixed.) For a loss of the decoded X at nh entries
 * (h_row[e], h_col[e]) with dloss/dX there = h_grad[e] (device arrays),
 * returns
 *   - dXt = dloss/dXt (rr x rc, leading dimension lddxt, device, FP32);
 *   - dLr, dLc: dloss/d(Laplacian values) on the CSR patterns (nnz FP64
 *     each, device, optional): nonzero only on the rows of unsampled nodes;
 *   - dwr, dwc: dloss/d(edge weights) (nnz FP32 each, optional; needs the
 *     weights wr, wc on the same patterns and lap_type), an undirected
 *     edge's derivative at both of its entries.
 * Same inputs and parameters as the forward call, plus the forward's k
 * (1 <= k <= kmax); the forward factors are recomputed with that k
 * (partial SVD, both upsampling solves), unless resume != 0: then `ws`
 * must be the workspace of a cpca_decode call with the same inputs and
 * parameters (cpca_decode accepts this larger workspace), whose factors are
 * reused (k must equal the k it found). Steps: scatter of h_grad into
 * dU, dV, dsigma; the adjoint of the column normalisation; one adjoint
 * Jacobi-PCG per side on L_aa (to cg_tol); the top-k SVD derivative
 * (Townsend's formula, with the parts outside the top-k subspaces through
 * the resolvents (s_i^2 I - Xt^T Xt)^-1 on the complement, solved by dense
 * CG on the Gram matrix of the shorter side, min(rr, rc) <= 16384).
 * The singular values s_1..s_k must be distinct and separated from s_{k+1}
 * (else CPCA_ERR_SINGULAR / CPCA_ERR_NOT_CONVERGED). SYNCHRONISES.
 * ---------------------------------------------------------------------- */
size_t cpca_decode_backward_workspace_size(int32_t p, int32_t n, int32_t rr, int32_t rc, int32_t kmax,
                                           int64_t nnz_r, int64_t nnz_c);
cpca_status cpca_decode_backward(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                 const int32_t* omega_r, const int32_t* omega_c, int32_t p, int32_t n,
                                 const cpca_csr* Lr, const cpca_csr* Lc,
                                 const cpca_decode_params* params, int32_t k, int32_t resume,
                                 int64_t nh,
                                 const int32_t* h_row, const int32_t* h_col, const float* h_grad,
                                 float* dXt, int64_t lddxt, double* dLr, double* dLc,
                                 const float* wr, const float* wc, int32_t lap_type, float* dwr,
                                 float* dwc, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Laplacians as functions of the edge weights (Sec. I), for differentiation.
 *
 * cpca_laplacian_values: on a given symmetric CSR pattern (pattern->val is
 * not read) with weights w (nnz FP32, 0 on the diagonal entries), writes
 * val (nnz FP32): D_i = sum_{j != i} w_ij (FP64); normalised
 * (CPCA_LAP_NORMALIZED): -w_ij / sqrt(D_i D_j) off the diagonal and 1 on it
 * (0 where D_i = 0); combinatorial: -w_ij and D_i. Asynchronous.
 * cpca_laplacian_weight_grad: the chain rule from dL = dloss/d(values)
 * (nnz FP64) to dw (nnz FP32) through that map, given the values L->val
 * and weights w; an undirected edge's derivative is written at both of its
 * entries, 0 on the diagonal. Asynchronous. Both need
 * cpca_laplacian_workspace_size(n) bytes of scratch.
 * ---------------------------------------------------------------------- */
size_t cpca_laplacian_workspace_size(int32_t n);
cpca_status cpca_laplacian_values(const cpca_csr* pattern, const float* w, int32_t lap_type, float* val,
                                  void* ws, size_t ws_bytes, void* stream);
cpca_status cpca_laplacian_weight_grad(const cpca_csr* L, const float* w, const double* dL,
                                       int32_t lap_type, float* dw, void* ws, size_t ws_bytes,
                                       void* stream);

/* cpca_decode_entries: X(h_row[e], h_col[e]) = sum_c U(i, c) sigma_c V(j, c)
 * (Algorithm 2 step 6 at nh given entries) from the U, V (ld columns) and
 * sigma that cpca_decode returns; FP64 sums, FP32 out. Asynchronous. */
cpca_status cpca_decode_entries(const float* U, const float* V, int32_t ld, const double* sigma,
                                int32_t k, int64_t nh, const int32_t* h_row, const int32_t* h_col,
                                float* out, void* stream);

/* ------------------------------------------------------------------------
 * cpca_cluster_decode - the clustering decoder (Sec. V-D, Algorithm 3).
 *
 * 1. k-means on the columns of Xt (rc points in R^rr): Lloyd's iteration
 *    from the k columns that the sampling generator picks on SplitMix64
 *    stream 5 with `seed` (ascending), nearest centre by squared Euclidean
 *    distance (ties: the lowest centre), centres the means of their points
 *    (an empty cluster keeps its centre), until an assignment step changes
 *    no label or after kmeans_iters steps (the paper leaves the start and
 *    the stop open);
 * 2. each column of C (n x k) is the minimiser of c^T L_c c subject to
 *    c(omega_c) = the one-hot k-means labels (Lemma 1), by Jacobi PCG to
 *    cg_tol (cg_max_iter <= 0: 10 x unsampled nodes);
 * 3. labels[i] = the column of row i's largest entry (ties: the lowest).
 * Xt: rr x rc (ldxt), omega_c: rc sampled columns of the n-node graph Lc
 * (ascending, distinct), all device. Outputs (device): labels (n int32);
 * optional labels_t (rc int32, the k-means labels) and C (n x k FP32).
 * 1 <= k <= min(48, rc). Workspace:
 * cpca_cluster_decode_workspace_size(rr, rc, n, k, nnz of Lc).
 * SYNCHRONISES. Returns CPCA_ERR_SINGULAR if a component of Lc holds no
 * sampled node, CPCA_ERR_NOT_CONVERGED if the PCG hit its cap (labels
 * still written), CPCA_ERR_TIMEOUT if a device barrier gave up.
 * ---------------------------------------------------------------------- */
typedef struct cpca_cluster_params {
  int32_t k;             /* clusters */
  int32_t kmeans_iters;  /* assignment steps at most (>= 1) */
  uint64_t seed;         /* initial centres */
  double cg_tol;         /* relative residual of the harmonic extension */
  int32_t cg_max_iter;
} cpca_cluster_params;

typedef struct cpca_cluster_info {
  int32_t kmeans_steps;  /* assignment steps taken */
  int32_t cg_iters;      /* largest PCG iteration count over the k columns */
  double cg_res;         /* largest final relative residual */
} cpca_cluster_info;

size_t cpca_cluster_decode_workspace_size(int32_t rr, int32_t rc, int32_t n, int32_t k, int64_t nnz_c);
cpca_status cpca_cluster_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt, const int32_t* omega_c,
                                int32_t n, const cpca_csr* Lc, const cpca_cluster_params* params,
                                int32_t* labels, int32_t* labels_t, float* C, cpca_cluster_info* info,
                                void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * cpca_subspace_project - the approximate decoders 2 and 3 (appendix,
 * "Other Approximate Decoders"): when the full data Y is available, only one
 * subspace is upsampled and X is a projection of Y:
 *   side 0 (decoder 2): X = U U^T Y, U the p x k upsampled, column-normalised
 *                       left basis (cpca_decode's U);
 *   side 1 (decoder 3): X = Y V V^T, V the n x k right basis (cpca_decode's V).
 * basis: device FP32, rows of ldb floats (ldb <= 48; cpca_decode's kmax),
 * first k columns used; Y p x n (ldy), X p x n (ldx), device FP32, X may not
 * alias Y. Workspace: cpca_subspace_project_workspace_size(p, n, ldb).
 * Asynchronous.
 * ---------------------------------------------------------------------- */
size_t cpca_subspace_project_workspace_size(int32_t p, int32_t n, int32_t ldb);
cpca_status cpca_subspace_project(int32_t side, const float* basis, int32_t ldb, int32_t k, const float* Y,
                                  int64_t ldy, int32_t p, int32_t n, float* X, int64_t ldx, void* ws,
                                  size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * cpca_alternate_decode - the alternate decoder (Sec. V-B,
 * Eq. alternatedecoder): the full p x n matrix X minimising
 *   |M_r X M_c - Xt|_F^2 + gamma_c tr(X L_c X^T) + gamma_r tr(X^T L_r X)
 * (gamma_r, gamma_c the paper's gamma-bars, user-chosen; Theorem 2 relates
 * them to a gamma and the graphs' spectral gaps), solved through its normal
 * equations D_r X D_c + gamma_c X L_c + gamma_r L_r X = M_r^T Xt M_c^T by
 * Jacobi-preconditioned conjugate gradients (the paper names CG for it,
 * cost O(I n p K)); D_r, D_c: 0/1 diagonals of the sampled rows/columns.
 *
 * Xt: rr x rc (leading dimension ldxt) FP32, device; omega_r (rr), omega_c
 * (rc): the sampled row/column indices (distinct, in range; Xt(a, b)
 * belongs to row omega_r[a], column omega_c[b]); Lr (p nodes), Lc (n
 * nodes): symmetric Laplacian CSR. X (p x n, ldx, device FP32) receives the
 * solution. x0 = 0; stops when |r|_2 <= tol |B|_2 or after max_iter
 * iterations. FP32 vectors, FP64 dot products. Workspace:
 * cpca_alternate_decode_workspace_size(p, n) bytes (six p x n FP32 arrays
 * and small tables). SYNCHRONISES (twice: index checks, result). Returns
 * CPCA_ERR_INVALID_ARG for bad or repeated omega entries,
 * CPCA_ERR_NOT_CONVERGED if max_iter was reached (X still written),
 * CPCA_ERR_TIMEOUT if a device barrier gave up.
 * ---------------------------------------------------------------------- */
typedef struct cpca_alt_params {
  double gamma_r;     /* weight of tr(X^T L_r X), >= 0 */
  double gamma_c;     /* weight of tr(X L_c X^T), >= 0 */
  double tol;         /* relative residual */
  int32_t max_iter;   /* CG iterations at most */
  int32_t blocks;     /* launch width cap; 0 = automatic */
} cpca_alt_params;

typedef struct cpca_alt_info {
  int32_t iters;
  int32_t converged;
  double rel_res;     /* |r|_2 / |B|_2 at the end */
} cpca_alt_info;

size_t cpca_alternate_decode_workspace_size(int32_t p, int32_t n);
cpca_status cpca_alternate_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                  const int32_t* omega_r, const int32_t* omega_c, int32_t p, int32_t n,
                                  const cpca_csr* Lr, const cpca_csr* Lc, const cpca_alt_params* params,
                                  float* X, int64_t ldx, cpca_alt_info* info, void* ws, size_t ws_bytes,
                                  void* stream);

/* ------------------------------------------------------------------------
 * cpca_kron_reduce - compressed Laplacian by Kron reduction (Sec. IV-A,
 * "Graphs for Compressed data"), the alternative to new kNN graphs on Y~:
 *   L~ = L(O, O) - L(O, Ob) L(Ob, Ob)^-1 L(Ob, O),
 * the Schur complement of the unsampled block Ob onto the sampled nodes O.
 * Column j of L~ is (L h_j)(O), h_j the harmonic extension (Lemma 1) of the
 * unit vector e_j given on O; the extensions are solved by the decoder's
 * Jacobi PCG, up to 48 columns per launch, to relative residual tol
 * (max_iter <= 0: 10 x unsampled nodes), and (L h_j)(O) is summed in FP64.
 * The result is symmetrised ((L~ + L~^T) / 2, the PCG leaves it symmetric
 * only to its tolerance). It is dense in general: two kept nodes are coupled
 * when a path joins them through unsampled nodes (Theorem III.4 of the
 * paper's reference on Kron reduction); entries with no such path are
 * exactly 0.
 *
 * L: symmetric Laplacian CSR on n nodes (normalised or combinatorial, the
 * reduction does not care), device; omega: rho sampled nodes, device int32,
 * strictly ascending, in [0, n) (checked: CPCA_ERR_INVALID_ARG); 1 <= rho
 * <= n. Lt: rho x rho FP32 row-major (leading dimension ldlt >= rho),
 * device, written. Optional rowptr (rho + 1 int64), col (rho^2 int32), val
 * (rho^2 FP32), device, all three or none: L~ again as CSR with every entry
 * stored, ready for cpca_frpcag_solve. Workspace:
 * cpca_kron_reduce_workspace_size(n, rho, nnz of L). SYNCHRONISES (once for
 * the index check, once per chunk of 48 columns). Returns CPCA_ERR_SINGULAR
 * if a connected component holds no sampled node (L(Ob, Ob) is singular),
 * CPCA_ERR_NOT_CONVERGED if a PCG column hit its cap (Lt still written),
 * CPCA_ERR_TIMEOUT if a device barrier gave up.
 * ---------------------------------------------------------------------- */
typedef struct cpca_kron_info {
  int32_t chunks;    /* PCG launches (ceil(rho / 48)) */
  int32_t cg_iters;  /* largest PCG iteration count over all columns */
  double cg_res;     /* largest final relative residual */
} cpca_kron_info;

size_t cpca_kron_reduce_workspace_size(int32_t n, int32_t rho, int64_t nnz);
cpca_status cpca_kron_reduce(const cpca_csr* L, const int32_t* omega, int32_t rho, double tol, int32_t max_iter,
                             float* Lt, int64_t ldlt, int64_t* rowptr, int32_t* col, float* val,
                             cpca_kron_info* info, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CPCA_H */
