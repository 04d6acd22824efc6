// fista.cu - FRPCAG on the sampled matrix by FISTA (Sec. IV-B,
// Eq. frpcag_small with phi = l1, Algorithm 1), the step size
// lambda = 1/beta' by power iteration, and the FP64 objective.
//
// One fused kernel per FISTA iteration. A block owns R consecutive rows:
// it stages Z_j(rows, :) in shared memory, forms (Z_j Lc)(rows, j) by
// shared-memory gathers along each column's Lc neighbour list (Lc is
// symmetric, so (Z Lc)_{ij} = sum_k Lc[j,k] Z_{ik}), forms (Lr Z_j)(i, j)
// from coalesced loads of the Lr-neighbour rows, then applies the gradient
// step, the l1 prox and the momentum update in registers and writes S_j
// (in place over S_{j-1}) and Z_{j+1}. Per iteration it reads Y~, S_{j-1},
// Z_j and writes S_j, Z_{j+1}: 20 bytes per entry of algorithmic traffic.
#include "common.cuh"
#include "fista_internal.cuh"

namespace cpca {
namespace {

// ------------------------------------------------------------- step size --
// Power iteration in FP64 on one Laplacian per block (block 0: Lr with
// stream 2, block 1: Lc with stream 3), then the Rayleigh quotient.
constexpr int PW_THREADS = 1024;

__device__ void spmv64(const CsrView& L, const double* __restrict__ v, double* __restrict__ w) {
  for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
    double s = 0.0;
    for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e) s += double(L.val[e]) * v[L.col[e]];
    w[i] = s;
  }
}

__global__ void __launch_bounds__(PW_THREADS)
power_kernel(CsrView Lr, CsrView Lc, int iters, uint64_t seed, double* __restrict__ vbuf,
             int vstride, double* __restrict__ out /* [norm_r, norm_c, lambda] */) {
  __shared__ double red[32];
  const CsrView L = blockIdx.x == 0 ? Lr : Lc;
  double* v = vbuf + int64_t(blockIdx.x) * 2 * vstride;
  double* w = v + vstride;
  const uint64_t s0 = stream_state0(seed, 2 + blockIdx.x);
  double ss = 0.0;
  for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
    const double x = uniform01_at(s0, uint64_t(i) + 1) - 0.5;
    v[i] = x;
    ss += x * x;
  }
  ss = block_sum(ss, red);
  double inv = ss > 0 ? 1.0 / sqrt(ss) : 0.0;
  for (int i = threadIdx.x; i < L.n; i += blockDim.x) v[i] *= inv;
  __syncthreads();
  bool zero = false;
  for (int it = 0; it < iters && !zero; ++it) {
    spmv64(L, v, w);
    double s = 0.0;
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) s += w[i] * w[i];
    s = block_sum(s, red);
    if (s == 0.0) {
      zero = true;
      break;
    }
    const double iw = 1.0 / sqrt(s);
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) v[i] = w[i] * iw;
    __syncthreads();
  }
  double lam = 0.0;
  if (!zero) {
    spmv64(L, v, w);
    __syncthreads();
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
      num += v[i] * w[i];
      den += v[i] * v[i];
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    lam = den > 0 ? num / den : 0.0;
  }
  if (threadIdx.x == 0) out[blockIdx.x] = lam;
}

__global__ void step_kernel(double gamma_r, double gamma_c, double step_given,
                            double* __restrict__ out /* [norm_r, norm_c, lambda] */) {
  if (threadIdx.x || blockIdx.x) return;
  if (step_given > 0) {
    out[2] = step_given;
    return;
  }
  const double beta = 2.0 * gamma_c * out[1] + 2.0 * gamma_r * out[0];
  out[2] = beta > 0 ? 1.0 / beta : 1.0;
}

// ------------------------------------------------------- FISTA iteration --
template <int R>
__global__ void __launch_bounds__(256)
fista_iter_kernel(const float* __restrict__ Yt, int64_t ldy, int rr, int rc, CsrView Lr,
                  CsrView Lc, const float* __restrict__ Zin, float* __restrict__ Zout,
                  float* __restrict__ S, int64_t lds, const double* __restrict__ lam_ptr,
                  float two_gr, float two_gc, float mu, int iter1, double eps,
                  const double* __restrict__ prev_stats, double* __restrict__ out_stats,
                  int* __restrict__ ctl) {
  extern __shared__ float zs[];  // [R][rc]
  __shared__ double red[8];
  // Device-side stop test of Algorithm 1: iteration j runs only if
  // iteration j-1 did not meet |Z_j - Z_{j-1}|^2 < eps |Z_{j-1}|^2.
  if (ctl[0]) return;
  if (prev_stats) {
    const double dz = prev_stats[0], nz = prev_stats[1];
    if (dz < eps * nz) {
      if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctl[0] = 1;
        ctl[1] = iter1 - 1;
      }
      return;
    }
  }
  const float lam = float(*lam_ptr);
  const int row0 = blockIdx.x * R;
  const int nrows = min(R, rr - row0);
  for (int r = 0; r < nrows; ++r)
    for (int j = threadIdx.x; j < rc; j += blockDim.x) zs[r * rc + j] = Zin[int64_t(row0 + r) * rc + j];
  __syncthreads();
  double dz = 0.0, nz = 0.0;
  for (int j = threadIdx.x; j < rc; j += blockDim.x) {
    float acc_c[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc_c[r] = 0.f;
    const int64_t e0 = Lc.rowptr[j], e1 = Lc.rowptr[j + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const int c = __ldg(Lc.col + e);
      const float w = __ldg(Lc.val + e);
#pragma unroll
      for (int r = 0; r < R; ++r) acc_c[r] = fmaf(w, zs[r * rc + c], acc_c[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= nrows) break;
      const int i = row0 + r;
      float acc_r = 0.f;
      const int64_t f0 = Lr.rowptr[i], f1 = Lr.rowptr[i + 1];
      for (int64_t f = f0; f < f1; ++f)
        acc_r = fmaf(__ldg(Lr.val + f), __ldg(Zin + int64_t(__ldg(Lr.col + f)) * rc + j), acc_r);
      const float z = zs[r * rc + j];
      const float g = fmaf(two_gr, acc_r, two_gc * acc_c[r]);
      const float v = fmaf(-lam, g, z);
      const float y = __ldg(Yt + int64_t(i) * ldy + j);
      const float dl = v - y;
      const float s = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
      const int64_t si = int64_t(i) * lds + j;
      const float sp = S[si];
      S[si] = s;
      const float zn = fmaf(mu, s - sp, s);
      Zout[int64_t(i) * rc + j] = zn;
      if (out_stats) {
        const double d = double(zn) - double(z);
        dz += d * d;
        nz += double(z) * double(z);
      }
    }
  }
  if (out_stats) {
    dz = block_sum(dz, red);
    nz = block_sum(nz, red);
    if (threadIdx.x == 0) {
      atomicAdd(out_stats, dz);
      atomicAdd(out_stats + 1, nz);
    }
  }
}

__global__ void init_kernel(const float* __restrict__ Yt, int64_t ldy, int rr, int rc,
                            float* __restrict__ Z, float* __restrict__ S, int64_t lds) {
  const int64_t total = int64_t(rr) * rc;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / rc), j = int(t % rc);
    const float y = Yt[int64_t(i) * ldy + j];
    Z[t] = y;
    S[int64_t(i) * lds + j] = y;
  }
}

// ------------------------------------------------------------- objective --
// F(X) = sum |Y~ - X| + gamma_c sum (X Lc) o X + gamma_r sum X o (Lr X), FP64,
// deterministic: fixed block partials summed in order by one block.
__global__ void objective_kernel(const float* __restrict__ Yt, int64_t ldy, int rr, int rc,
                                 CsrView Lr, CsrView Lc, const float* __restrict__ X, int64_t ldx,
                                 double gr, double gc, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = blockIdx.x; i < rr; i += gridDim.x) {
    for (int j = threadIdx.x; j < rc; j += blockDim.x) {
      const double x = X[int64_t(i) * ldx + j];
      double xl = 0.0, lx = 0.0;
      for (int64_t e = Lc.rowptr[j]; e < Lc.rowptr[j + 1]; ++e)
        xl += double(Lc.val[e]) * double(X[int64_t(i) * ldx + Lc.col[e]]);
      for (int64_t f = Lr.rowptr[i]; f < Lr.rowptr[i + 1]; ++f)
        lx += double(Lr.val[f]) * double(X[int64_t(Lr.col[f]) * ldx + j]);
      acc += fabs(double(Yt[int64_t(i) * ldy + j]) - x) + gc * xl * x + gr * x * lx;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
__global__ void sum_in_order_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  *out = s;
}

constexpr int OBJ_BLOCKS = 512;

}  // namespace

FistaWs fista_layout(void* ws, int rr, int rc, int max_iter_stats) {
  Carve c(ws);
  FistaWs w{};
  w.Z0 = c.take<float>(size_t(rr) * rc);
  w.Z1 = c.take<float>(size_t(rr) * rc);
  w.scal = c.take<double>(4);
  w.vbuf = c.take<double>(size_t(4) * std::max(rr, rc));
  w.stats = c.take<double>(size_t(2) * std::max(max_iter_stats, 1));
  w.ctl = c.take<int>(4);
  w.part = c.take<double>(OBJ_BLOCKS);
  w.obj = c.take<double>(1);
  w.bytes = c.bytes();
  return w;
}

cpca_status power_step(const CsrView& Lr, const CsrView& Lc, int iters, uint64_t seed,
                       double gamma_r, double gamma_c, double step_given, const FistaWs& w,
                       cudaStream_t st) {
  if (step_given <= 0) {
    CPCA_PROF("power_iter", st);
    power_kernel<<<2, PW_THREADS, 0, st>>>(Lr, Lc, iters, seed, w.vbuf, std::max(Lr.n, Lc.n),
                                            w.scal);
    CPCA_LAUNCHED();
  } else {
    CPCA_CUDA(cudaMemsetAsync(w.scal, 0, 2 * sizeof(double), st));
  }
  step_kernel<<<1, 32, 0, st>>>(gamma_r, gamma_c, step_given, w.scal);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

int fista_rows_per_block(int rc) {
  const int64_t budget = 96 * 1024;
  const int64_t per_row = int64_t(rc) * 4;
  if (per_row * 8 <= budget) return 8;
  if (per_row * 4 <= budget) return 4;
  if (per_row * 2 <= budget) return 2;
  return 1;
}

template <int R>
static cpca_status launch_iter(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                               const CsrView& Lc, const float* Zin, float* Zout, float* S,
                               int64_t lds, const double* lam, float two_gr, float two_gc,
                               float mu, int iter1, double eps, const double* prev_stats,
                               double* out_stats, int* ctl, cudaStream_t st) {
  const size_t smem = size_t(R) * rc * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    CPCA_CUDA(cudaFuncSetAttribute(fista_iter_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
    attr_set = true;
  }
  const int threads = rc >= 256 ? 256 : ((rc + 31) / 32) * 32;
  CPCA_PROF("fista_iter", st);
  fista_iter_kernel<R><<<ceil_div(rr, R), threads, smem, st>>>(
      Yt, ldy, rr, rc, Lr, Lc, Zin, Zout, S, lds, lam, two_gr, two_gc, mu, iter1, eps, prev_stats,
      out_stats, ctl);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status fista_iteration(int R, const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* Zin, float* Zout, float* S,
                            int64_t lds, const double* lam, double gamma_r, double gamma_c,
                            double mu, int iter1, double eps, const double* prev_stats,
                            double* out_stats, int* ctl, cudaStream_t st) {
  const float tr = float(2.0 * gamma_r), tc = float(2.0 * gamma_c), m = float(mu);
  switch (R) {
    case 8: return launch_iter<8>(Yt, ldy, rr, rc, Lr, Lc, Zin, Zout, S, lds, lam, tr, tc, m, iter1, eps, prev_stats, out_stats, ctl, st);
    case 4: return launch_iter<4>(Yt, ldy, rr, rc, Lr, Lc, Zin, Zout, S, lds, lam, tr, tc, m, iter1, eps, prev_stats, out_stats, ctl, st);
    case 2: return launch_iter<2>(Yt, ldy, rr, rc, Lr, Lc, Zin, Zout, S, lds, lam, tr, tc, m, iter1, eps, prev_stats, out_stats, ctl, st);
    default: return launch_iter<1>(Yt, ldy, rr, rc, Lr, Lc, Zin, Zout, S, lds, lam, tr, tc, m, iter1, eps, prev_stats, out_stats, ctl, st);
  }
}

cpca_status fista_init(const float* Yt, int64_t ldy, int rr, int rc, float* Z, float* S,
                       int64_t lds, cudaStream_t st) {
  const unsigned blocks = std::min<unsigned>(ceil_div(int64_t(rr) * rc, 256), num_sms() * 8);
  init_kernel<<<blocks, 256, 0, st>>>(Yt, ldy, rr, rc, Z, S, lds);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            const FistaWs& w, cudaStream_t st) {
  CPCA_PROF("fista_objective", st);
  objective_kernel<<<OBJ_BLOCKS, 256, 0, st>>>(Yt, ldy, rr, rc, Lr, Lc, X, ldx, gr, gc, w.part);
  CPCA_LAUNCHED();
  sum_in_order_kernel<<<1, 32, 0, st>>>(w.part, OBJ_BLOCKS, w.obj);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

// Momentum coefficients mu_j = (t_j - 1) / t_{j+1} of Algorithm 1, t_1 = 1.
void fista_momentum(int J, double* mu) {
  double t = 1.0;
  for (int j = 0; j < J; ++j) {
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    mu[j] = (t - 1.0) / tn;
    t = tn;
  }
}

cpca_status check_csr(const cpca_csr* L, int n, const char* name) {
  if (!L || !L->rowptr || (L->nnz > 0 && (!L->col || !L->val))) {
    set_error("%s: null CSR pointer", name);
    return CPCA_ERR_INVALID_ARG;
  }
  if (L->n != n || L->nnz < 0) {
    set_error("%s: CSR has n=%d, expected %d", name, L->n, n);
    return CPCA_ERR_INVALID_ARG;
  }
  return CPCA_OK;
}

}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_frpcag_workspace_size(int32_t rr, int32_t rc) {
  if (rr <= 0 || rc <= 0) return 0;
  return fista_layout(nullptr, rr, rc, kMaxStatIters).bytes;
}

extern "C" cpca_status cpca_frpcag_solve(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                         const cpca_csr* Lr, const cpca_csr* Lc,
                                         const cpca_frpcag_params* prm, float* X, int64_t ldx,
                                         cpca_solve_info* info, void* ws, size_t ws_bytes,
                                         void* stream) {
  clear_error();
  CPCA_CHECK_ARG(Yt && X && prm, "cpca_frpcag_solve: null pointer");
  CPCA_CHECK_ARG(rr > 0 && rc > 0, "cpca_frpcag_solve: empty matrix");
  CPCA_CHECK_ARG(ldyt >= rc && ldx >= rc, "cpca_frpcag_solve: leading dimension too small");
  CPCA_CHECK_ARG(prm->max_iter >= 0, "cpca_frpcag_solve: max_iter < 0");
  CPCA_CHECK_ARG(prm->gamma_r >= 0 && prm->gamma_c >= 0, "cpca_frpcag_solve: negative gamma");
  CPCA_CHECK_ARG(prm->eps >= 0, "cpca_frpcag_solve: eps < 0");
  CPCA_CHECK_ARG(prm->step > 0 || prm->power_iters >= 1, "cpca_frpcag_solve: power_iters < 1");
  CPCA_CHECK_ARG(prm->eps == 0 || prm->check_every >= 1, "cpca_frpcag_solve: check_every < 1");
  CPCA_CHECK_ARG(int64_t(rc) * 4 <= 200 * 1024, "cpca_frpcag_solve: rc too large for one row in shared memory");
  CPCA_TRY(check_csr(Lr, rr, "cpca_frpcag_solve(Lr)"));
  CPCA_TRY(check_csr(Lc, rc, "cpca_frpcag_solve(Lc)"));
  const FistaWs w = fista_layout(ws, rr, rc, kMaxStatIters);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_frpcag_solve: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const CsrView lr{Lr->n, Lr->rowptr, Lr->col, Lr->val};
  const CsrView lc{Lc->n, Lc->rowptr, Lc->col, Lc->val};
  const int J = prm->max_iter;
  CPCA_TRY(power_step(lr, lc, prm->power_iters, prm->power_seed, prm->gamma_r, prm->gamma_c,
                      prm->step, w, st));
  CPCA_TRY(fista_init(Yt, ldyt, rr, rc, w.Z0, X, ldx, st));
  CPCA_CUDA(cudaMemsetAsync(w.ctl, 0, 4 * sizeof(int), st));
  const bool want = prm->eps > 0 || info != nullptr;
  const int nstat = std::min(J, kMaxStatIters);
  if (want && nstat > 0) CPCA_CUDA(cudaMemsetAsync(w.stats, 0, 2 * sizeof(double) * nstat, st));
  CPCA_CHECK_ARG(prm->eps == 0 || J <= kMaxStatIters, "cpca_frpcag_solve: eps > 0 needs max_iter <= %d",
                 kMaxStatIters);
  std::vector<double> mu(std::max(J, 1));
  fista_momentum(J, mu.data());
  const int R = fista_rows_per_block(rc);
  int done_iters = J;
  for (int j = 1; j <= J; ++j) {
    const float* Zin = (j & 1) ? w.Z0 : w.Z1;
    float* Zout = (j & 1) ? w.Z1 : w.Z0;
    // statistics: slot j-1 for every iteration when eps > 0 (iteration j
    // tests slot j-2), else slot 0 for the last iteration only
    const double* prev = (prm->eps > 0 && j > 1) ? w.stats + 2 * (j - 2) : nullptr;
    double* out = prm->eps > 0 ? w.stats + 2 * (j - 1) : ((info && j == J) ? w.stats : nullptr);
    CPCA_TRY(fista_iteration(R, Yt, ldyt, rr, rc, lr, lc, Zin, Zout, X, ldx, w.scal + 2,
                             prm->gamma_r, prm->gamma_c, mu[j - 1], j, prm->eps, prev, out, w.ctl,
                             st));
    if (prm->eps > 0 && (j % prm->check_every == 0) && j < J) {
      int ctl[2];
      CPCA_CUDA(cudaMemcpyAsync(ctl, w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
      CPCA_CUDA(cudaStreamSynchronize(st));
      if (ctl[0]) break;
    }
  }
  if (info) {
    CPCA_TRY(fista_objective(Yt, ldyt, rr, rc, lr, lc, X, ldx, prm->gamma_r, prm->gamma_c, w, st));
    int ctl[2];
    double scal[3], obj, last[2] = {0, 0};
    CPCA_CUDA(cudaMemcpyAsync(ctl, w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(scal, w.scal, sizeof(scal), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&obj, w.obj, sizeof(obj), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));
    if (ctl[0]) done_iters = ctl[1];
    if (done_iters > 0) {
      const int s = prm->eps > 0 ? done_iters - 1 : 0;
      CPCA_CUDA(cudaMemcpy(last, w.stats + 2 * s, sizeof(last), cudaMemcpyDeviceToHost));
    }
    info->iters = done_iters;
    info->norm_r = scal[0];
    info->norm_c = scal[1];
    info->step = scal[2];
    info->rel_change = last[1] > 0 ? last[0] / last[1] : 0.0;
    info->objective = obj;
  }
  return CPCA_OK;
}
