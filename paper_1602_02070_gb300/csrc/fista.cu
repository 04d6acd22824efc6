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
// Power iteration on both Laplacians in one cooperative launch (warp per
// row, rows of Lr then Lc), then the Rayleigh quotients and lambda.
// With v_k = u_k / |u_k| the iteration v <- L v / |L v| is carried as
// u_{k+1} = (L u_k) / |u_k|, so each step needs one grid barrier (for
// |u_{k+1}|). Start vector u_0(i) = SplitMix64 uniform - 1/2 (stream 2 for
// Lr, 3 for Lc). Iterates FP32, norms and quotients FP64.
struct PowerArgs {
  CsrView L[2];
  int iters;
  uint64_t seed;
  float* u[2][2];      // [graph][ping/pong]
  double* acc;         // ring [3][2]: |u|^2 per graph
  double* fin;         // [2][2]: u^T L u, u^T u per graph
  double gamma_r, gamma_c, step_given;
  double* out;         // [norm_r, norm_c, lambda]
  GridBar bar;
};

__device__ __forceinline__ double warp_red_add(double v) { return warp_sum(v); }

__global__ void __launch_bounds__(512)
power_persistent_kernel(PowerArgs a) {
  __shared__ double sacc[2];
  const int lane = threadIdx.x & 31;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n0 = a.L[0].n, rows = n0 + a.L[1].n;
  if (threadIdx.x < 2) sacc[threadIdx.x] = 0.0;
  __syncthreads();
  // u_0 and |u_0|^2 into ring slot 0
  for (int r = wid * 32 + lane; r < rows; r += nwarp * 32) {
    const int g = r < n0 ? 0 : 1, i = g ? r - n0 : r;
    const double x = uniform01_at(stream_state0(a.seed, 2 + g), uint64_t(i) + 1) - 0.5;
    a.u[g][0][i] = float(x);
    atomicAdd(&sacc[g], x * x);
  }
  __syncthreads();
  if (threadIdx.x < 2 && sacc[threadIdx.x] != 0.0) atomicAdd(a.acc + threadIdx.x, sacc[threadIdx.x]);
  if (!grid_sync(a.bar)) return;
  double nrm2[2] = {__ldcg(a.acc), __ldcg(a.acc + 1)};
  bool zero[2] = {!(nrm2[0] > 0), !(nrm2[1] > 0)};
  for (int k = 0; k < a.iters; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    if (threadIdx.x < 2) sacc[threadIdx.x] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x < 2) a.acc[2 * ((k + 2) % 3) + threadIdx.x] = 0.0;
    __syncthreads();
    const float inv[2] = {zero[0] ? 0.f : float(1.0 / sqrt(nrm2[0])), zero[1] ? 0.f : float(1.0 / sqrt(nrm2[1]))};
    for (int r = wid; r < rows; r += nwarp) {
      const int g = r < n0 ? 0 : 1, i = g ? r - n0 : r;
      const CsrView& L = a.L[g];
      const float* u = a.u[g][cur];
      float sum = 0.f;
      for (int64_t e = L.rowptr[i] + lane; e < L.rowptr[i + 1]; e += 32)
        sum = fmaf(__ldg(L.val + e), __ldcg(u + __ldg(L.col + e)), sum);
      sum = warp_sumf(sum) * inv[g];
      if (lane == 0) {
        a.u[g][nxt][i] = sum;
        atomicAdd(&sacc[g], double(sum) * double(sum));
      }
    }
    __syncthreads();
    double* slot = a.acc + 2 * ((k + 1) % 3);
    if (threadIdx.x < 2 && sacc[threadIdx.x] != 0.0) atomicAdd(slot + threadIdx.x, sacc[threadIdx.x]);
    if (!grid_sync(a.bar)) return;
    for (int g = 0; g < 2; ++g) {
      if (zero[g]) continue;
      nrm2[g] = __ldcg(slot + g);
      if (!(nrm2[g] > 0)) zero[g] = true;
    }
  }
  // Rayleigh quotients u^T L u / u^T u of the final iterate
  const int fin = a.iters & 1;
  __shared__ double snum[2], sden[2];
  if (threadIdx.x < 2) {
    snum[threadIdx.x] = 0.0;
    sden[threadIdx.x] = 0.0;
  }
  __syncthreads();
  for (int r = wid; r < rows; r += nwarp) {
    const int g = r < n0 ? 0 : 1, i = g ? r - n0 : r;
    const CsrView& L = a.L[g];
    const float* u = a.u[g][fin];
    float sum = 0.f;
    for (int64_t e = L.rowptr[i] + lane; e < L.rowptr[i + 1]; e += 32)
      sum = fmaf(__ldg(L.val + e), __ldcg(u + __ldg(L.col + e)), sum);
    sum = warp_sumf(sum);
    if (lane == 0) {
      const double ui = __ldcg(u + i);
      atomicAdd(&snum[g], ui * double(sum));
      atomicAdd(&sden[g], ui * ui);
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    atomicAdd(a.fin + 2 * threadIdx.x, snum[threadIdx.x]);
    atomicAdd(a.fin + 2 * threadIdx.x + 1, sden[threadIdx.x]);
  }
  if (!grid_sync(a.bar)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double nr[2];
    for (int g = 0; g < 2; ++g) {
      const double num = __ldcg(a.fin + 2 * g), den = __ldcg(a.fin + 2 * g + 1);
      nr[g] = (zero[g] || !(den > 0)) ? 0.0 : num / den;
    }
    a.out[0] = nr[0];
    a.out[1] = nr[1];
    if (a.step_given > 0) {
      a.out[2] = a.step_given;
    } else {
      const double beta = 2.0 * a.gamma_c * nr[1] + 2.0 * a.gamma_r * nr[0];
      a.out[2] = beta > 0 ? 1.0 / beta : 1.0;
    }
  }
}

__global__ void step_kernel(double step_given, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  out[0] = 0.0;
  out[1] = 0.0;
  out[2] = step_given;
}

// ------------------------------------------------------- FISTA iteration --
// Persistent form: all J iterations in one cooperative launch, one bounded
// grid barrier per iteration. The matrix is cut into 32 x 32 tiles. Z_j is
// kept twice, row-major (Z) and column-major (ZT = Z_j^T), so that both
// graph products read contiguous 128-byte segments:
//   (Lr Z)(i, j)  = sum_k Lr[i, k] Z(k, j)    -> segments of rows of Z,
//   (Z Lc)(i, j)  = sum_k Lc[j, k] ZT(k, i)   -> segments of rows of ZT
// (Lc is symmetric). A tile stages the 32 neighbour lists of its rows (Lr)
// and of its columns (Lc) in shared memory, so each list is read once per
// tile, not once per row. Warps batch NB neighbour loads for each of their
// 4 rows (or columns) before consuming any. Z_j is read through L2
// (ld.global.cg) because other blocks wrote it during the previous
// iteration of this launch.
constexpr int TB = 32;        // tile edge
constexpr int kTileNbr = 40;  // neighbour-list entries staged per row / column

struct FistaPersistArgs {
  const float* Yt;
  int64_t ldy;
  int rr, rc;
  CsrView Lr, Lc;
  float* Z[2];    // row-major Z_j ping / pong (ld rc)
  float* ZT[2];   // column-major copies (ld rr)
  float* S;
  int64_t lds;
  const double* lam;
  float two_gr, two_gc;
  int J;
  double eps;
  double* stats;     // ring [4][2]: slot j % 4 holds iteration j's sums
  int want_last;     // accumulate statistics of the last iteration
  int* ctl;          // [stopped, iterations]
  GridBar bar;
};

struct TileSmem {
  int64_t roff[TB][kTileNbr];  // element offset of neighbour row k in Z  (k * rc)
  float rval[TB][kTileNbr];
  int64_t coff[TB][kTileNbr];  // element offset of neighbour row k in ZT (k * rr)
  float cval[TB][kTileNbr];
  float ac[TB][TB + 1];     // (Z Lc) of the tile, [row][col]
  float zt[TB][TB + 1];     // Z_{j+1} tile for the transposed store, [row][col]
  int rdeg[TB], cdeg[TB];
  int64_t rf0[TB], cf0[TB];
};

// For four staged neighbour lists u = 0..3 (rows or columns of the tile):
// out[u] = sum_q w[u][q] * x[off[u][q] + base]. Chunks of 8 entries of all
// four lists are loaded together (32 independent loads per lane) up to the
// shortest list, then each list's remainder, then entries beyond the
// staging area straight from the CSR.
__device__ __forceinline__ void nbr_sum4(const int64_t (*off)[kTileNbr], const float (*w)[kTileNbr],
                                         const int* deg, const int64_t* f0, int first, bool valid,
                                         const float* __restrict__ x, int64_t base, const CsrView& L,
                                         int64_t stride, float out[4]) {
  int dmin = kTileNbr;
#pragma unroll
  for (int u = 0; u < 4; ++u) dmin = min(dmin, min(deg[first + u], kTileNbr));
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (valid) {
    int e = 0;
    for (; e + 8 <= dmin; e += 8) {
      float v[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 8; ++q) v[u][q] = __ldcg(x + off[first + u][e + q] + base);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[u] = fmaf(w[first + u][e + q], v[u][q], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ds = min(deg[first + u], kTileNbr);
      int e2 = e;
      for (; e2 + 4 <= ds; e2 += 4) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldcg(x + off[first + u][e2 + q] + base);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[u] = fmaf(w[first + u][e2 + q], v[q], acc[u]);
      }
      for (; e2 < ds; ++e2) acc[u] = fmaf(w[first + u][e2], __ldcg(x + off[first + u][e2] + base), acc[u]);
      for (int64_t f = f0[first + u] + kTileNbr; f < f0[first + u] + deg[first + u]; ++f)
        acc[u] = fmaf(__ldg(L.val + f), __ldcg(x + int64_t(__ldg(L.col + f)) * stride + base), acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] = acc[u];
}

// RESIDENT: every block owns at most one tile for the whole solve; its
// neighbour lists are staged once, and Y~, S and the tile's own Z_j entries
// stay in registers across iterations (S is written back at the end).
// Otherwise blocks stream over tiles, staging lists per tile.
__device__ __forceinline__ void stage_tile(TileSmem& sm, const FistaPersistArgs& a, int i0, int j0,
                                           int ni, int nj) {
  if (threadIdx.x < TB) {
    const int r = threadIdx.x;
    const int64_t f0 = r < ni ? a.Lr.rowptr[i0 + r] : 0;
    sm.rf0[r] = f0;
    sm.rdeg[r] = r < ni ? int(a.Lr.rowptr[i0 + r + 1] - f0) : 0;
  } else if (threadIdx.x < 2 * TB) {
    const int c = threadIdx.x - TB;
    const int64_t g0 = c < nj ? a.Lc.rowptr[j0 + c] : 0;
    sm.cf0[c] = g0;
    sm.cdeg[c] = c < nj ? int(a.Lc.rowptr[j0 + c + 1] - g0) : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * kTileNbr; e += blockDim.x) {
    const int r = e / kTileNbr, q = e % kTileNbr;
    if (q < min(sm.rdeg[r], kTileNbr)) {
      sm.roff[r][q] = int64_t(__ldg(a.Lr.col + sm.rf0[r] + q)) * a.rc;
      sm.rval[r][q] = __ldg(a.Lr.val + sm.rf0[r] + q);
    }
    if (q < min(sm.cdeg[r], kTileNbr)) {
      sm.coff[r][q] = int64_t(__ldg(a.Lc.col + sm.cf0[r] + q)) * a.rr;
      sm.cval[r][q] = __ldg(a.Lc.val + sm.cf0[r] + q);
    }
  }
  __syncthreads();
}

template <bool RESIDENT>
__global__ void __launch_bounds__(256, RESIDENT ? 5 : 4)
fista_persistent_kernel(FistaPersistArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(smraw);
  __shared__ double red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float lam = float(*a.lam);
  const int nti = (a.rr + TB - 1) / TB, ntj = (a.rc + TB - 1) / TB;
  const int ntiles = nti * ntj;
  // resident state (one tile per block)
  float ry[4], rs[4], rz[4];
  int ri0 = 0, rj0 = 0, rni = 0, rnj = 0;
  if (RESIDENT && blockIdx.x < ntiles) {
    ri0 = (blockIdx.x / ntj) * TB;
    rj0 = (blockIdx.x % ntj) * TB;
    rni = min(TB, a.rr - ri0);
    rnj = min(TB, a.rc - rj0);
    stage_tile(sm, a, ri0, rj0, rni, rnj);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = warp * 4 + u;
      const bool in = r < rni && lane < rnj;
      const int64_t i = ri0 + r, jj = rj0 + lane;
      ry[u] = in ? a.Yt[i * a.ldy + jj] : 0.f;
      rs[u] = ry[u];  // S_0 = Y~
      rz[u] = ry[u];  // Z_1 = Y~
    }
  }
  int done = a.J;
  double t = 1.0;  // t_j of Algorithm 1 (t_1 = 1)
  for (int j = 1; j <= a.J; ++j) {
    if (a.eps > 0 && j > 1) {
      const double* ps = a.stats + 2 * ((j - 1) & 3);
      if (__ldcg(ps) < a.eps * __ldcg(ps + 1)) {
        done = j - 1;
        break;
      }
    }
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const float mu = float((t - 1.0) / tn);
    t = tn;
    const float* Zin = a.Z[(j - 1) & 1];
    const float* ZTin = a.ZT[(j - 1) & 1];
    float* Zout = a.Z[j & 1];
    float* ZTout = a.ZT[j & 1];
    const bool stats = a.eps > 0 || (a.want_last && j == a.J);
    double* st = a.stats + 2 * (j & 3);
    // slot (j + 1) % 4 was last read at the start of iteration j - 2
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.stats[2 * ((j + 1) & 3)] = 0.0;
      a.stats[2 * ((j + 1) & 3) + 1] = 0.0;
    }
    double dz = 0.0, nz = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      int i0, j0, ni, nj;
      if (RESIDENT) {
        i0 = ri0; j0 = rj0; ni = rni; nj = rnj;
      } else {
        i0 = (tile / ntj) * TB;
        j0 = (tile % ntj) * TB;
        ni = min(TB, a.rr - i0);
        nj = min(TB, a.rc - j0);
        stage_tile(sm, a, i0, j0, ni, nj);
      }
      // (Z Lc): warp w takes tile columns 4w..4w+3, lane = tile row
      {
        float o[4];
        nbr_sum4(sm.coff, sm.cval, sm.cdeg, sm.cf0, warp * 4, lane < ni, ZTin, i0 + lane, a.Lc,
                 a.rr, o);
#pragma unroll
        for (int u = 0; u < 4; ++u) sm.ac[lane][warp * 4 + u] = o[u];
      }
      // (Lr Z): warp w takes tile rows 4w..4w+3, lane = tile column
      float ar[4];
      nbr_sum4(sm.roff, sm.rval, sm.rdeg, sm.rf0, warp * 4, lane < nj, Zin, j0 + lane, a.Lr, a.rc, ar);
      __syncthreads();  // sm.ac complete
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = warp * 4 + u;
        if (r < ni && lane < nj) {
          const int64_t i = i0 + r, jj = j0 + lane;
          const float z = RESIDENT ? rz[u] : __ldcg(Zin + i * a.rc + jj);
          const float y = RESIDENT ? ry[u] : __ldg(a.Yt + i * a.ldy + jj);
          const float sp = RESIDENT ? rs[u] : a.S[i * a.lds + jj];
          const float gr = fmaf(a.two_gr, ar[u], a.two_gc * sm.ac[r][lane]);
          const float v = fmaf(-lam, gr, z);
          const float dl = v - y;
          const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
          const float zn = fmaf(mu, sv - sp, sv);
          if (RESIDENT) {
            rs[u] = sv;
            rz[u] = zn;
          } else {
            a.S[i * a.lds + jj] = sv;
          }
          Zout[i * a.rc + jj] = zn;
          sm.zt[r][lane] = zn;
          if (stats) {
            const double d = double(zn) - double(z);
            dz += d * d;
            nz += double(z) * double(z);
          }
        }
      }
      __syncthreads();  // sm.zt complete
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = warp * 4 + u;
        if (c < nj && lane < ni) ZTout[int64_t(j0 + c) * a.rr + i0 + lane] = sm.zt[lane][c];
      }
      if (!RESIDENT) __syncthreads();  // before the next tile reuses shared memory
    }
    if (stats) {
      dz = block_sum(dz, red);
      nz = block_sum(nz, red);
      if (threadIdx.x == 0) {
        atomicAdd(st, dz);
        atomicAdd(st + 1, nz);
      }
    }
    if (!grid_sync(a.bar)) return;
  }
  if (RESIDENT && blockIdx.x < ntiles) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = warp * 4 + u;
      if (r < rni && lane < rnj) a.S[int64_t(ri0 + r) * a.lds + rj0 + lane] = rs[u];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl[0] = done < a.J ? 1 : 0;
    a.ctl[1] = done;
  }
}

// Z_1 = S_0 = Y~ (Algorithm 1), plus the transposed copy of Z_1.
__global__ void init_kernel(const float* __restrict__ Yt, int64_t ldy, int rr, int rc,
                            float* __restrict__ Z, float* __restrict__ ZT, float* __restrict__ S,
                            int64_t lds) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < rr && j < rc) {
      const float y = Yt[int64_t(i) * ldy + j];
      Z[int64_t(i) * rc + j] = y;
      S[int64_t(i) * lds + j] = y;
      tile[r][threadIdx.x] = y;
    }
  }
  __syncthreads();
  if (ZT)
    for (int c = threadIdx.y; c < 32; c += blockDim.y) {
      const int j = j0 + c, i = i0 + threadIdx.x;
      if (i < rr && j < rc) ZT[int64_t(j) * rr + i] = tile[threadIdx.x][c];
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


}  // namespace

FistaWs fista_layout(void* ws, int rr, int rc, int /*unused*/) {
  Carve c(ws);
  FistaWs w{};
  w.Z0 = c.take<float>(size_t(rr) * rc);
  w.Z1 = c.take<float>(size_t(rr) * rc);
  w.ZT0 = c.take<float>(size_t(rr) * rc);
  w.ZT1 = c.take<float>(size_t(rr) * rc);
  w.scal = c.take<double>(4);
  for (int g = 0; g < 2; ++g)
    for (int b = 0; b < 2; ++b) w.pu[g][b] = c.take<float>(size_t(g ? rc : rr) + 4);
  w.pacc = c.take<double>(6 + 4);
  w.stats = c.take<double>(8);
  w.ctl = c.take<int>(4);
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.part = c.take<double>(kObjBlocks);
  w.obj = c.take<double>(1);
  w.bytes = c.bytes();
  return w;
}

static int coop_blocks(const void* kernel, int threads, size_t smem, int want) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  return std::max(1, std::min(want, std::max(occ, 1) * num_sms()));
}

cpca_status power_step(const CsrView& Lr, const CsrView& Lc, int iters, uint64_t seed,
                       double gamma_r, double gamma_c, double step_given, const FistaWs& w,
                       cudaStream_t st) {
  if (step_given > 0) {
    step_kernel<<<1, 32, 0, st>>>(step_given, w.scal);
    CPCA_LAUNCHED();
    return CPCA_OK;
  }
  PowerArgs a{};
  a.L[0] = Lr;
  a.L[1] = Lc;
  a.iters = iters;
  a.seed = seed;
  for (int g = 0; g < 2; ++g)
    for (int b = 0; b < 2; ++b) a.u[g][b] = w.pu[g][b];
  a.acc = w.pacc;
  a.fin = w.pacc + 6;
  a.gamma_r = gamma_r;
  a.gamma_c = gamma_c;
  a.step_given = step_given;
  a.out = w.scal;
  a.bar = GridBar{w.bar, w.bar + kBarrierCounters, w.err};
  CPCA_CUDA(cudaMemsetAsync(w.pacc, 0, sizeof(double) * 10, st));
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  const int rows = Lr.n + Lc.n;
  // one warp per row, at most one 512-thread block per SM (fewer arrivals
  // at the per-iteration grid barrier)
  const int grid = std::min(num_sms(), coop_blocks((const void*)power_persistent_kernel, 512, 0,
                                                   (rows + 15) / 16));
  void* args[] = {&a};
  CPCA_PROF("power_iter", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)power_persistent_kernel, dim3(grid), dim3(512),
                                        args, 0, st));
  CPCA_LAUNCHED();
  return CPCA_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// All J iterations of Algorithm 1 in one cooperative launch.
cpca_status fista_run(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                      const CsrView& Lc, float* X, int64_t ldx, double gamma_r, double gamma_c,
                      int J, double eps, bool want_last, int tile_rows, const FistaWs& w,
                      cudaStream_t st) {
  (void)tile_rows;
  CPCA_TRY(fista_init(Yt, ldy, rr, rc, w.Z0, w.ZT0, X, ldx, st));
  CPCA_CUDA(cudaMemsetAsync(w.stats, 0, 8 * sizeof(double), st));
  CPCA_CUDA(cudaMemsetAsync(w.ctl, 0, 4 * sizeof(int), st));
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  if (J == 0) return CPCA_OK;
  FistaPersistArgs a{};
  a.Yt = Yt;
  a.ldy = ldy;
  a.rr = rr;
  a.rc = rc;
  a.Lr = Lr;
  a.Lc = Lc;
  a.Z[0] = w.Z0;
  a.Z[1] = w.Z1;
  a.ZT[0] = w.ZT0;
  a.ZT[1] = w.ZT1;
  a.S = X;
  a.lds = ldx;
  a.lam = w.scal + 2;
  a.two_gr = float(2.0 * gamma_r);
  a.two_gc = float(2.0 * gamma_c);
  a.J = J;
  a.eps = eps;
  a.stats = w.stats;
  a.want_last = want_last ? 1 : 0;
  a.ctl = w.ctl;
  a.bar = GridBar{w.bar, w.bar + kBarrierCounters, w.err};
  const size_t smem = sizeof(TileSmem);
  const int tiles = int(ceil_div(rr, TB) * int64_t(ceil_div(rc, TB)));
  const void* kres = (const void*)fista_persistent_kernel<true>;
  const void* kstr = (const void*)fista_persistent_kernel<false>;
  CPCA_CUDA(cudaFuncSetAttribute(kres, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  CPCA_CUDA(cudaFuncSetAttribute(kstr, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int cap_res = coop_blocks(kres, 256, smem, 1 << 30);
  const bool resident = tiles <= cap_res;
  const void* kern = resident ? kres : kstr;
  const int grid = resident ? tiles : coop_blocks(kstr, 256, smem, tiles);
  void* args[] = {&a};
  CPCA_PROF("fista_persistent", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(256), args, smem, st));
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status fista_init(const float* Yt, int64_t ldy, int rr, int rc, float* Z, float* ZT, float* S,
                       int64_t lds, cudaStream_t st) {
  dim3 grid(ceil_div(rc, 32), ceil_div(rr, 32)), block(32, 8);
  init_kernel<<<grid, block, 0, st>>>(Yt, ldy, rr, rc, Z, ZT, S, lds);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            const FistaWs& w, cudaStream_t st) {
  CPCA_PROF("fista_objective", st);
  objective_kernel<<<kObjBlocks, 256, 0, st>>>(Yt, ldy, rr, rc, Lr, Lc, X, ldx, gr, gc, w.part);
  CPCA_LAUNCHED();
  sum_in_order_kernel<<<1, 32, 0, st>>>(w.part, kObjBlocks, w.obj);
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
  CPCA_CHECK_ARG(prm->tile_rows == 0 || prm->tile_rows == 1 || prm->tile_rows == 2 ||
                     prm->tile_rows == 4 || prm->tile_rows == 8,
                 "cpca_frpcag_solve: tile_rows must be 0, 1, 2, 4 or 8");
  CPCA_CHECK_ARG(prm->step > 0 || prm->power_iters >= 1, "cpca_frpcag_solve: power_iters < 1");
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
  CPCA_TRY(fista_run(Yt, ldyt, rr, rc, lr, lc, X, ldx, prm->gamma_r, prm->gamma_c, J, prm->eps,
                     info != nullptr, prm->tile_rows, w, st));
  int done_iters = J;
  if (info) {
    CPCA_TRY(fista_objective(Yt, ldyt, rr, rc, lr, lc, X, ldx, prm->gamma_r, prm->gamma_c, w, st));
    int ctl[2];
    double scal[3], obj, ring[8];
    int err = 0;
    CPCA_CUDA(cudaMemcpyAsync(ctl, w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(scal, w.scal, sizeof(scal), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&obj, w.obj, sizeof(obj), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(ring, w.stats, sizeof(ring), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));
    if (err) {
      set_error("cpca_frpcag_solve: grid barrier timed out");
      return CPCA_ERR_TIMEOUT;
    }
    if (J > 0) done_iters = ctl[1];
    const double* last = ring + 2 * (done_iters & 3);
    info->iters = done_iters;
    info->norm_r = scal[0];
    info->norm_c = scal[1];
    info->step = scal[2];
    info->rel_change = done_iters > 0 && last[1] > 0 ? last[0] / last[1] : 0.0;
    info->objective = obj;
  }
  return CPCA_OK;
}
