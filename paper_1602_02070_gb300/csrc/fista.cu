// fista.cu - FRPCAG on the sampled matrix by FISTA (Sec. IV-B,
// Eq. frpcag_small with phi = l1, Algorithm 1), the step size
// lambda = 1/beta' by power iteration, and the FP64 objective.
//
// Everything runs over an instance table (a single solve is a batch of
// one; the batched entry point takes up to kMaxBatch independent problems of
// different sizes, gammas and graphs). The table travels by value in the
// kernel parameters, so a solve makes no host round trip and can be
// captured in a CUDA graph.
//
//   power_batch_kernel   all power iterations of all Laplacians, one
//                        cooperative launch, one grid barrier per step
//   step_kernel          lambda per instance
//   init_batch_kernel    Z_1 = S_0 = Y~ and the transposed copy of Z_1
//   fista_batch_kernel   all J iterations of every instance, one cooperative
//                        launch, one grid barrier per iteration
//
// FISTA data layout: the matrix of each instance is cut into 32 x 32 tiles
// listed one after another across instances. Z_j is kept twice, row-major
// (Z) and column-major (ZT = Z_j^T), so that both graph products read
// contiguous 128-byte segments:
//   (Lr Z)(i, j) = sum_k Lr[i, k] Z(k, j)   -> segments of rows of Z,
//   (Z Lc)(i, j) = sum_k Lc[j, k] ZT(k, i)  -> segments of rows of ZT
// (Lc is symmetric). A tile stages the neighbour lists of its 32 rows (Lr)
// and 32 columns (Lc) in shared memory. Z_j is read through L2
// (ld.global.cg) because other blocks wrote it during the previous
// iteration of the same launch. Algorithmic traffic per iteration: read Y~,
// S_{j-1}, Z_j and write S_j, Z_{j+1}: 20 bytes per entry.
#include <cmath>
#include <cooperative_groups.h>
#include <memory>
#include <map>
#include <type_traits>
#include <mutex>

#include "common.cuh"
#include "fista_internal.cuh"

namespace cpca {
namespace {

// ------------------------------------------------------------- step size --
// Power iteration on a list of Laplacians (two per instance: Lr with stream
// 2, Lc with stream 3), then the Rayleigh quotients. With v_k = u_k / |u_k|
// the iteration v <- L v / |L v| is carried as u_{k+1} = (L u_k) / |u_k|, so
// each step needs one synchronisation (for |u_{k+1}|). Start vector
// u_0(i) = SplitMix64 uniform - 1/2. Iterates FP32, norms and quotients
// FP64; the scale 1/|u_k| only keeps the iterate bounded (the quotient does
// not depend on it) and is taken in FP32 (FP64 square roots sit on every
// step's critical path).
//
// Arithmetic shared by both kernels below (so that a graph's estimate does
// not depend on the kernel, the launch or the other graphs): one thread per
// row, each graph's rows padded to whole warps ("warp blocks", graph g's
// first at w0); (L u)(i) by FMAs in CSR order; each warp block's FP64 sum
// of squares; a graph's |u|^2 the sum of its warp blocks' sums, lane-strided
// in block order then a butterfly (the same bits in every lane).
struct PowerGraph {
  CsrView L;
  double* out;  // |L|_2 estimate
  int stream;
  int w0;       // first warp block in the warp-padded row list
  // kept iterates for reverse mode (null in a plain solve)
  float* U;               // [(T + 1) * n]: u_t at U + t * n
  double* nrm2;           // [T + 1]: |u_t|^2
  float* Ub;              // [T * n]: ubar_t at Ub + (t - 1) * n
  const double* rho_bar;  // d loss / d rho
};
struct PowerBatchArgs {
  PowerGraph g[2 * kMaxBatch];
  int ngraph;
  int iters;
  uint64_t seed;
  GridBar bar;
};

__device__ __forceinline__ int find_graph_warp(const PowerBatchArgs& a, int vw) {
  int lo = 0, hi = a.ngraph - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.g[mid].w0 <= vw) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// sum over graph G's warp blocks of part[w0 + w] (see above); CG: through L2
template <bool CG = false>
__device__ __forceinline__ double graph_warp_sum(const double* part, const PowerGraph& G, int lane) {
  const int nw = (G.L.n + 31) >> 5;
  double t = 0.0;
  for (int w = lane; w < nw; w += 32) t += CG ? __ldcg(part + G.w0 + w) : part[G.w0 + w];
  return warp_sum(t);
}

// Grid-wide version for graph sets larger than one cluster: every warp of a
// cooperative launch takes warp blocks in turn; the iterate (padded row
// order, ping-pong) and the warp-block sums live in global scratch; one grid
// barrier per step. Kept iterates (G.U) as in the cluster kernel.
__global__ void __launch_bounds__(512)
power_batch_kernel(const __grid_constant__ PowerBatchArgs a, int nvw, float* __restrict__ u,
                   double* __restrict__ wq, double* __restrict__ rq) {
  const int lane = threadIdx.x & 31;
  const int nwt = (gridDim.x * blockDim.x) >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int NV = 32 * nvw;
  for (int vw = gw; vw < nvw; vw += nwt) {
    const PowerGraph& G = a.g[find_graph_warp(a, vw)];
    const int i = (vw - G.w0) * 32 + lane;
    double q = 0.0;
    float x0 = 0.f;
    if (i < G.L.n) {
      const double x = uniform01_at(stream_state0(a.seed, G.stream), uint64_t(i) + 1) - 0.5;
      q = x * x;
      x0 = float(x);
      if (G.U) G.U[i] = x0;
    }
    u[vw * 32 + lane] = x0;
    q = warp_sum(q);
    if (lane == 0) wq[vw] = q;
  }
  if (!grid_sync(a.bar)) return;
  auto spmv = [&](const PowerGraph& G, int i, const float* x) {
    const int vbase = 32 * G.w0;
    float acc = 0.f;
    for (int64_t e = G.L.rowptr[i]; e < G.L.rowptr[i + 1]; ++e)
      acc = fmaf(__ldg(G.L.val + e), __ldcg(x + vbase + __ldg(G.L.col + e)), acc);
    return acc;
  };
  for (int k = 0; k < a.iters; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    for (int vw = gw; vw < nvw; vw += nwt) {
      const PowerGraph& G = a.g[find_graph_warp(a, vw)];
      const int i = (vw - G.w0) * 32 + lane;
      const double n2 = graph_warp_sum<true>(wq + cur * nvw, G, lane);
      if (G.nrm2 && vw == G.w0 && lane == 0) G.nrm2[k] = n2;
      const float inv = n2 > 0 ? rsqrtf(float(n2)) : 0.f;  // only the direction matters
      const float s = i < G.L.n ? spmv(G, i, u + cur * NV) * inv : 0.f;
      if (i < G.L.n && G.U) G.U[size_t(k + 1) * G.L.n + i] = s;
      u[nxt * NV + vw * 32 + lane] = s;
      const double q = warp_sum(double(s) * double(s));
      if (lane == 0) wq[nxt * nvw + vw] = q;
    }
    if (!grid_sync(a.bar)) return;
  }
  // Rayleigh quotients u^T L u / u^T u of the final iterate
  const int fin = a.iters & 1;
  for (int vw = gw; vw < nvw; vw += nwt) {
    const PowerGraph& G = a.g[find_graph_warp(a, vw)];
    const int i = (vw - G.w0) * 32 + lane;
    const float* x = u + fin * NV;
    const float lu = i < G.L.n ? spmv(G, i, x) : 0.f;
    const double ui = i < G.L.n ? double(__ldcg(x + vw * 32 + lane)) : 0.0;
    const double num = warp_sum(ui * double(lu)), den = warp_sum(ui * ui);
    if (lane == 0) {
      rq[vw] = num;
      rq[nvw + vw] = den;
    }
  }
  if (!grid_sync(a.bar)) return;
  if (blockIdx.x == 0)
    for (int g = threadIdx.x >> 5; g < a.ngraph; g += blockDim.x >> 5) {
      const PowerGraph& H = a.g[g];
      const double nm = graph_warp_sum<true>(rq, H, lane), dn = graph_warp_sum<true>(rq + nvw, H, lane);
      const double last = graph_warp_sum<true>(wq + fin * nvw, H, lane);
      if (lane == 0) {
        *H.out = (dn > 0 && last > 0) ? nm / dn : 0.0;
        if (H.nrm2) H.nrm2[a.iters] = last;
      }
    }
}

// The same power iterations for graph sets that one thread-block cluster
// holds: each graph's rows padded to whole warps, at most kPowMaxWarps warps
// in all. One thread per row. A CTA keeps its rows' CSR entries in shared
// memory as a sliced ELL block per warp (entry e of lane l at e * 32 + l, so
// a warp's loads hit distinct banks); entries beyond the shared budget come
// from the CSR arrays. Every CTA holds the whole iterate (padded row order,
// ping-pong), and each new entry, like each warp's FP64 sum of squares, is
// written into all CTAs through distributed shared memory; one cluster
// barrier per iteration orders it. A graph's |u|^2 is the sum of its warps'
// partials in warp order, taken identically by every warp, so the result
// does not depend on the launch shape or on the other graphs of the batch.
constexpr int kPowCtas = 8;
constexpr int kPowMaxWarps = kPowCtas * 32;

// One thread's row in the one-cluster kernels: its graph, its CSR row and the
// warp's sliced-ELL block in shared memory (min(longest row of the warp,
// equal share of the budget) slots; padding entries are (0, 0.0)).
struct PowRow {
  const PowerGraph* G;
  int vw, i, vbase, deg, slots, lane;
  bool wact, valid;
  int64_t e0;
  const int2* el;

  __device__ __forceinline__ void init(const PowerBatchArgs& a, int nvw, int2* ell, int ell_cap,
                                       int crank, int nctas = kPowCtas) {
    lane = threadIdx.x & 31;
    const int lw = threadIdx.x >> 5, nlw = blockDim.x >> 5;
    vw = lw * nctas + crank;
    wact = vw < nvw;
    G = &a.g[wact ? find_graph_warp(a, vw) : 0];
    i = (vw - G->w0) * 32 + lane;
    valid = wact && i < G->L.n;
    vbase = 32 * G->w0;
    e0 = 0;
    deg = 0;
    if (valid) {
      e0 = G->L.rowptr[i];
      deg = int(G->L.rowptr[i + 1] - e0);
    }
    slots = deg;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) slots = max(slots, __shfl_xor_sync(0xffffffffu, slots, o));
    const int dcap = ell_cap / (32 * nlw);
    slots = min(slots, dcap);
    int2* mine = ell + size_t(lw) * dcap * 32 + lane;
    for (int e = 0; e < slots; ++e)
      mine[e * 32] =
          e < deg ? make_int2(vbase + G->L.col[e0 + e], __float_as_int(G->L.val[e0 + e])) : make_int2(0, 0);
    el = mine;
  }
  // (L x)(i), x in padded row order; CSR order, one FMA per entry
  __device__ __forceinline__ float spmv(const float* x) const {
    float acc = 0.f;
#pragma unroll 4
    for (int e = 0; e < slots; ++e) {
      const int2 v = el[e * 32];
      acc = fmaf(__int_as_float(v.y), x[v.x], acc);
    }
    for (int e = slots; e < deg; ++e)
      acc = fmaf(__ldg(G->L.val + e0 + e), x[vbase + __ldg(G->L.col + e0 + e)], acc);
    return acc;
  }
};

// lane l of a warp sends float4 chunk (l & 7) of the warp's 32 values to
// CTAs (l >> 3) and (l >> 3) + 4 of the cluster, at float offset off0 there
__device__ __forceinline__ void allgather32(float v, float* xr0, float* xr1, int off0, int lane) {
  const int ch = lane & 7;
  float4 v4;
  v4.x = __shfl_sync(0xffffffffu, v, 4 * ch);
  v4.y = __shfl_sync(0xffffffffu, v, 4 * ch + 1);
  v4.z = __shfl_sync(0xffffffffu, v, 4 * ch + 2);
  v4.w = __shfl_sync(0xffffffffu, v, 4 * ch + 3);
  *reinterpret_cast<float4*>(xr0 + off0 + 4 * ch) = v4;
  *reinterpret_cast<float4*>(xr1 + off0 + 4 * ch) = v4;
}

// Forward, on a cluster of C CTAs (8, or 16 where the device allows that
// non-portable cluster size; the launch sets the cluster shape). With G.U
// set, also keeps u_0..u_T and |u_t|^2 (reverse mode).
template <int C>
__global__ void __launch_bounds__(1024)
power_cluster_kernel(const __grid_constant__ PowerBatchArgs a, int nvw, int ell_cap) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = int(cl.block_rank());
  extern __shared__ __align__(16) unsigned char smraw[];
  const int NV = 32 * nvw;
  double* wq = reinterpret_cast<double*>(smraw);  // [2][nvw]: warp sums of u_k^2
  double* rq = wq + 2 * nvw;                      // [2][nvw]: warp sums of u^T L u, u^T u
  float* xv = reinterpret_cast<float*>(rq + 2 * nvw);  // [2][NV]: the iterate
  int2* ell = reinterpret_cast<int2*>(xv + 2 * NV);
  PowRow R;
  R.init(a, nvw, ell, ell_cap, crank, C);
  const PowerGraph& G = *R.G;
  const int lane = R.lane, lw = threadIdx.x >> 5, nlw = blockDim.x >> 5, vw = R.vw;
  // u_0 and the warp sums of its squares (FP64, before rounding), computed
  // alike in every CTA
  for (int r = threadIdx.x; r < NV; r += blockDim.x) {
    const PowerGraph& H = a.g[find_graph_warp(a, r >> 5)];
    const int j = r - 32 * H.w0;
    xv[r] = j < H.L.n ? float(uniform01_at(stream_state0(a.seed, H.stream), uint64_t(j) + 1) - 0.5) : 0.f;
  }
  for (int w = lw; w < nvw; w += nlw) {
    const PowerGraph& H = a.g[find_graph_warp(a, w)];
    const int j = (w - H.w0) * 32 + lane;
    double q = 0.0;
    if (j < H.L.n) {
      const double x = uniform01_at(stream_state0(a.seed, H.stream), uint64_t(j) + 1) - 0.5;
      q = x * x;
    }
    q = warp_sum(q);
    if (lane == 0) wq[w] = q;
  }
  if (R.valid && G.U)
    G.U[R.i] = float(uniform01_at(stream_state0(a.seed, G.stream), uint64_t(R.i) + 1) - 0.5);
  // lane l sends float4 chunk (l & 7) of its warp's values to CTAs
  // (l >> 3) + 4 t, t < C / 4, and its warp sum to CTA l % C
  float* xr[C / 4];
#pragma unroll
  for (int t = 0; t < C / 4; ++t) xr[t] = cl.map_shared_rank(xv, (lane >> 3) + 4 * t);
  double* wr = cl.map_shared_rank(wq, lane & (C - 1));
  cl.sync();  // all CTAs running and initialised before any remote write
  for (int k = 0; k < a.iters; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    if (R.wact) {
      const double n2 = graph_warp_sum(wq + cur * nvw, G, lane);
      if (G.nrm2 && vw == G.w0 && lane == 0) G.nrm2[k] = n2;
      const float inv = n2 > 0 ? rsqrtf(float(n2)) : 0.f;  // only the direction matters
      const float s = R.valid ? R.spmv(xv + cur * NV) * inv : 0.f;
      if (R.valid && G.U) G.U[size_t(k + 1) * G.L.n + R.i] = s;
      {
        const int ch = lane & 7;
        float4 v4;
        v4.x = __shfl_sync(0xffffffffu, s, 4 * ch);
        v4.y = __shfl_sync(0xffffffffu, s, 4 * ch + 1);
        v4.z = __shfl_sync(0xffffffffu, s, 4 * ch + 2);
        v4.w = __shfl_sync(0xffffffffu, s, 4 * ch + 3);
#pragma unroll
        for (int t = 0; t < C / 4; ++t) *reinterpret_cast<float4*>(xr[t] + nxt * NV + vw * 32 + 4 * ch) = v4;
      }
      const double q = warp_sum(double(s) * double(s));
      if (lane < C) wr[nxt * nvw + vw] = q;
    }
    cl.sync();
  }
  // Rayleigh quotients u^T L u / u^T u of the final iterate, gathered in CTA 0
  const int fin = a.iters & 1;
  if (R.wact) {
    const float* x = xv + fin * NV;
    const float lu = R.valid ? R.spmv(x) : 0.f;
    const double u = R.valid ? double(x[vw * 32 + lane]) : 0.0;
    const double num = warp_sum(u * double(lu)), den = warp_sum(u * u);
    double* r0 = cl.map_shared_rank(rq, 0);
    if (lane == 0) r0[vw] = num;
    if (lane == 1) r0[nvw + vw] = den;
  }
  cl.sync();
  if (crank == 0)
    for (int g = lw; g < a.ngraph; g += nlw) {
      const PowerGraph& H = a.g[g];
      const double nm = graph_warp_sum(rq, H, lane), dn = graph_warp_sum(rq + nvw, H, lane);
      const double last = graph_warp_sum(wq + fin * nvw, H, lane);
      if (lane == 0) {
        *H.out = (dn > 0 && last > 0) ? nm / dn : 0.0;
        if (H.nrm2) H.nrm2[a.iters] = last;
      }
    }
}

// Reverse mode of the kept power iterations (rho = u_T^T L u_T / u_T^T u_T,
// v_t = u_t / |u_t|): vbar_T = 2 rhobar (L v_T - rho v_T), then for
// t = T..1 with d_t = v_t^T vbar_t
//   ubar_t = (vbar_t - d_t v_t) / |u_t|,
//   vbar_{t-1} = L ubar_t = (L vbar_t - d_t L v_t) / |u_t|,
// where L v_t is the forward's u_{t+1} (t < T). Carrying vbar instead of
// ubar lets one all-gather and one cluster barrier serve each step: vbar_t
// and the warp partials of d_t travel together. ubar_t goes to G.Ub for the
// Laplacian's own derivative.
__global__ void __cluster_dims__(kPowCtas, 1, 1) __launch_bounds__(1024)
power_cluster_reverse_kernel(const __grid_constant__ PowerBatchArgs a, int nvw, int ell_cap) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int crank = int(cl.block_rank());
  extern __shared__ __align__(16) unsigned char smraw[];
  const int NV = 32 * nvw;
  double* dq = reinterpret_cast<double*>(smraw);       // [2][nvw]: warp sums of v_t vbar_t
  float* xv = reinterpret_cast<float*>(dq + 4 * nvw);  // [2][NV]: vbar_t
  int2* ell = reinterpret_cast<int2*>(xv + 2 * NV);
  PowRow R;
  R.init(a, nvw, ell, ell_cap, crank);
  const PowerGraph& G = *R.G;
  const int lane = R.lane, vw = R.vw, T = a.iters, n = G.L.n;
  // u_T (from the tape) into the buffer that vbar_{T-1} takes later
  float* ut = xv + ((T + 1) & 1) * NV;
  for (int r = threadIdx.x; r < NV; r += blockDim.x) {
    const PowerGraph& H = a.g[find_graph_warp(a, r >> 5)];
    const int j = r - 32 * H.w0;
    ut[r] = j < H.L.n ? H.U[size_t(T) * H.L.n + j] : 0.f;
  }
  __syncthreads();
  float* xr0 = cl.map_shared_rank(xv, lane >> 3);
  float* xr1 = cl.map_shared_rank(xv, (lane >> 3) + 4);
  double* wr = cl.map_shared_rank(dq, lane & 7);
  auto inv_norm = [&](int t) {
    const double n2 = G.nrm2[t];
    return n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
  };
  double lvt = 0.0;  // (L v_t)(i) for t = T
  cl.sync();  // all CTAs running before any remote write
  if (R.wact) {
    const double invT = inv_norm(T);
    const double lu = R.valid ? double(R.spmv(ut)) : 0.0;
    const double vi = R.valid ? double(ut[vw * 32 + lane]) * invT : 0.0;
    lvt = lu * invT;
    const float vb = R.valid ? float(2.0 * (*G.rho_bar) * (lvt - (*G.out) * vi)) : 0.f;
    allgather32(vb, xr0, xr1, (T & 1) * NV + vw * 32, lane);
    const double q = warp_sum(vi * double(vb));
    if (lane < kPowCtas) wr[(T & 1) * nvw + vw] = q;
  }
  cl.sync();
  for (int t = T; t >= 1; --t) {
    const int cur = t & 1, nxt = cur ^ 1;
    if (R.wact) {
      const double d = graph_warp_sum(dq + cur * nvw, G, lane);
      const double inv = inv_norm(t);
      const double vb = R.valid ? double(xv[cur * NV + vw * 32 + lane]) : 0.0;
      const double vt = R.valid ? double(G.U[size_t(t) * n + R.i]) * inv : 0.0;
      if (R.valid) G.Ub[size_t(t - 1) * n + R.i] = float((vb - vt * d) * inv);
      if (t > 1) {
        const double lvb = R.valid ? double(R.spmv(xv + cur * NV)) : 0.0;
        const double lv = t == T ? lvt : (R.valid ? double(G.U[size_t(t + 1) * n + R.i]) : 0.0);
        const float vbm = R.valid ? float((lvb - d * lv) * inv) : 0.f;
        const double vm = R.valid ? double(G.U[size_t(t - 1) * n + R.i]) * inv_norm(t - 1) : 0.0;
        allgather32(vbm, xr0, xr1, nxt * NV + vw * 32, lane);
        const double q = warp_sum(vm * double(vbm));
        if (lane < kPowCtas) wr[nxt * nvw + vw] = q;
      }
    }
    if (t > 1) cl.sync();
  }
}

// lambda = 1/beta', beta' = 2 gamma_c |Lc|_2 + 2 gamma_r |Lr|_2 (or the given
// step); with beta' = 0 the smooth part vanishes and lambda = 1.
struct StepArgs {
  double* scal[kMaxBatch];  // [|Lr|, |Lc|, lambda]
  double gamma_r[kMaxBatch], gamma_c[kMaxBatch], step[kMaxBatch];
  int n;
};
__global__ void step_kernel(const __grid_constant__ StepArgs a) {
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    double* s = a.scal[i];
    if (a.step[i] > 0) {
      s[0] = 0.0;
      s[1] = 0.0;
      s[2] = a.step[i];
    } else {
      const double beta = 2.0 * a.gamma_c[i] * s[1] + 2.0 * a.gamma_r[i] * s[0];
      s[2] = beta > 0 ? 1.0 / beta : 1.0;
    }
  }
}

// ------------------------------------------------------- FISTA iteration --
// mu_j = (t_j - 1) / t_{j+1}, t_1 = 1, t_{j+1} = (1 + sqrt(1 + 4 t_j^2)) / 2
// (Algorithm 1): the same numbers for every solve, computed once on the host
// in FP64 (IEEE +, *, / and sqrt round identically there and here) and kept
// in constant memory; c_t_last = t_kMuTable continues the recurrence.
constexpr int kMuTable = 8192;
__constant__ float c_mu[kMuTable];
__constant__ double c_t_last;

struct FistaInst {
  const float* Yt;
  float* S;
  float* Z[2];   // row-major Z_j ping / pong (ld ldz = rc rounded up to 4)
  float* ZT[2];  // column-major copies (ld ldzt = rr rounded up to 4)
  CsrView Lr, Lc;
  const double* lam;
  double* stats;  // ring [4][2]: slot j % 4 holds iteration j's |dZ|^2, |Z|^2
  int* done;      // [stopped, iterations]
  int64_t ldy, lds;
  int64_t ldz, ldzt;
  float two_gr, two_gc;
  int rr, rc;
  int tile0, ntj;  // first tile in the batch list, column tiles
  int yvec, svec;  // Y~ / S rows allow 16-byte loads (ld % 4 == 0, aligned)
};
struct FistaBatchArgs {
  FistaInst in[kMaxBatch];
  int ninst;
  int ntiles;
  int J;
  double eps;
  int want_last;
  GridBar bar;
  // warm start (single problems): iterations 1..j0 done before, S holds
  // S_{j0}, warm_prev S_{j0-1}; mu0 = mu_{j0}, t0 = t_{j0+1}. prev_out
  // (optional) receives S_{J-1} of this call.
  int j0;
  const float* warm_prev;
  float* prev_out;
  int pvec;  // prev_out rows allow 16-byte stores
  float mu0;
  double t0;
};

__device__ __forceinline__ int find_inst(const FistaBatchArgs& a, int tile) {
  int lo = 0, hi = a.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.in[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename Off>
struct TileSmemT {
  TileNbrT<Off> nb;            // neighbour lists of the tile's rows and columns
  float ac[TB][TB + 1];        // (Z Lc) of the tile, [row][col]
  float zt[TB][TB + 1];        // Z_{j+1} tile for the transposed store, [row][col]
  unsigned int stopped[kMaxBatch / 32];
  float mu;                    // momentum coefficient of the iteration
};
using TileSmem = TileSmemT<int64_t>;
using TileSmem32 = TileSmemT<int32_t>;  // resident launches (tiles below 2^31 entries)

template <typename Off>
__device__ __forceinline__ void stage_tile(TileSmemT<Off>& sm, const FistaInst& I, int i0, int j0, int ni,
                                           int nj) {
  stage_nbr(sm.nb, I.Lr, I.Lc, int(I.ldzt), int(I.ldz), i0, j0, ni, nj);
}

// Four consecutive entries of a row (t < n valid), one 16-byte access when
// the row allows it.
__device__ __forceinline__ float4 load4(const float* p, bool vec, int n) {
  if (vec) return *reinterpret_cast<const float4*>(p);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (n > 0) v.x = p[0];
  if (n > 1) v.y = p[1];
  if (n > 2) v.z = p[2];
  if (n > 3) v.w = p[3];
  return v;
}
__device__ __forceinline__ void store4(float* p, float4 v, bool vec, int n) {
  if (vec) {
    *reinterpret_cast<float4*>(p) = v;
    return;
  }
  if (n > 0) p[0] = v.x;
  if (n > 1) p[1] = v.y;
  if (n > 2) p[2] = v.z;
  if (n > 3) p[3] = v.w;
}
__device__ __forceinline__ float& comp(float4& v, int t) {
  return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}

// RESIDENT: every block owns at most one tile for the whole solve; its
// neighbour lists are staged once and S stays in registers across
// iterations (written back at the end); Y~ and the tile's own Z_j come
// through L2 like the neighbours.
// Otherwise blocks stream over the tile list, staging lists per tile.
// Thread layout: lane group g = lane / 8 of warp w owns tile row
// r = 4 w + g (and, for the column products and the transposed store, tile
// column r); its 8 lanes own 4 consecutive columns (rows) each, read and
// written as 16-byte vectors (Z, ZT rows padded to multiples of 4).
// Stopping rule (eps > 0): instance i stops after iteration j - 1 once
// |Z_j - Z_{j-1}|^2 < eps |Z_{j-1}|^2; its tiles are then skipped, and the
// launch ends when no instance is left.
template <bool RESIDENT>
__global__ void __launch_bounds__(256, RESIDENT ? 5 : 4)
fista_batch_kernel(const __grid_constant__ FistaBatchArgs a) {
  using Off = typename std::conditional<RESIDENT, int32_t, int64_t>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  TileSmemT<Off>& sm = *reinterpret_cast<TileSmemT<Off>*>(smraw);
  __shared__ double red[8];
  __shared__ int any_active;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = warp * 4 + (lane >> 3);  // tile row (column) of this lane group
  const int cq = 4 * (lane & 7);          // first of the lane's 4 tile columns (rows)
  // resident state (one tile per block): S in registers
  float4 rs = make_float4(0.f, 0.f, 0.f, 0.f);
  int rinst = 0, ri0 = 0, rj0 = 0, rni = 0, rnj = 0;
  if (RESIDENT && blockIdx.x < a.ntiles) {
    rinst = find_inst(a, blockIdx.x);
    const FistaInst& I = a.in[rinst];
    const int lt = blockIdx.x - I.tile0;
    ri0 = (lt / I.ntj) * TB;
    rj0 = (lt % I.ntj) * TB;
    rni = min(TB, I.rr - ri0);
    rnj = min(TB, I.rc - rj0);
    stage_tile(sm, I, ri0, rj0, rni, rnj);
    if (rl < rni && cq < rnj)
      rs = a.warm_prev ? load4(I.S + int64_t(ri0 + rl) * I.lds + rj0 + cq, I.svec, rnj - cq)  // S_{j0}
                       : load4(I.Yt + int64_t(ri0 + rl) * I.ldy + rj0 + cq, I.yvec, rnj - cq);  // S_0 = Y~
  }
  double t = 1.0;  // t_j of Algorithm 1 (t_1 = 1)
  int jlast = a.J;
  if (threadIdx.x < kMaxBatch / 32) sm.stopped[threadIdx.x] = 0u;
  __syncthreads();
  for (int j = 1; j <= a.J; ++j) {
    // which instances run iteration j (with a fixed count, all of them)
    if (a.eps > 0) {
      if (threadIdx.x < kMaxBatch / 32) sm.stopped[threadIdx.x] = 0u;
      if (threadIdx.x == 0) any_active = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < a.ninst; i += blockDim.x) {
        const FistaInst& I = a.in[i];
        bool stop = __ldcg(I.done) != 0;
        if (!stop && j > 1) {
          const double* ps = I.stats + 2 * ((j - 1) & 3);
          stop = __ldcg(ps) < a.eps * __ldcg(ps + 1);
          // the block owning the instance's first tile records the count once
          if (stop && blockIdx.x == I.tile0 % gridDim.x) {
            I.done[1] = j - 1;
            I.done[0] = 1;
          }
        }
        if (stop) atomicOr(&sm.stopped[i >> 5], 1u << (i & 31));
        else any_active = 1;
      }
      __syncthreads();
      if (!any_active) {
        jlast = j - 1;
        break;
      }
    }
    // mu_jg of the global iteration jg = j0 + j from the table; beyond it,
    // t_{jg+1} in FP64 by one thread (from the table's end, or from t0 when
    // a resumed solve starts beyond it)
    const int jg = a.j0 + j;
    float mu;
    if (jg < kMuTable) {
      mu = c_mu[jg];
    } else {
      if (threadIdx.x == 0) {
        if (jg == kMuTable) t = c_t_last;
        else if (j == 1) t = a.t0;
        const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        sm.mu = float((t - 1.0) / tn);
        t = tn;
      }
      __syncthreads();
      mu = sm.mu;
    }
    const bool stats = a.eps > 0 || (a.want_last && j == a.J);
    // slot (j + 1) % 4 was last read at the start of iteration j - 2
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < a.ninst; i += blockDim.x) {
        a.in[i].stats[2 * ((j + 1) & 3)] = 0.0;
        a.in[i].stats[2 * ((j + 1) & 3) + 1] = 0.0;
      }
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      const int ii = RESIDENT ? rinst : find_inst(a, tile);
      if ((sm.stopped[ii >> 5] >> (ii & 31)) & 1u) continue;
      const FistaInst& I = a.in[ii];
      const float* Zin = I.Z[(j - 1) & 1];
      const float* ZTin = I.ZT[(j - 1) & 1];
      float* Zout = I.Z[j & 1];
      float* ZTout = I.ZT[j & 1];
      const float lam = float(*I.lam);
      int i0, j0, ni, nj;
      if (RESIDENT) {
        i0 = ri0; j0 = rj0; ni = rni; nj = rnj;
      } else {
        // column-block-major order: the tiles in flight at one time share
        // few column blocks of Z (the row products' gathers stay in L2)
        const int lt = tile - I.tile0, nti = (I.rr + TB - 1) / TB;
        i0 = (lt % nti) * TB;
        j0 = (lt / nti) * TB;
        ni = min(TB, I.rr - i0);
        nj = min(TB, I.rc - j0);
        stage_tile(sm, I, i0, j0, ni, nj);
      }
      // (Z Lc): column rl of the tile, rows cq..cq+3 (from ZT)
      {
        const float4 o = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.coff[rl], sm.nb.cval[rl], sm.nb.cdeg[rl], sm.nb.cf0[rl],
                                    rl < nj && cq < ni, ZTin, i0 + cq, I.Lc, I.ldzt);
        sm.ac[cq][rl] = o.x;
        sm.ac[cq + 1][rl] = o.y;
        sm.ac[cq + 2][rl] = o.z;
        sm.ac[cq + 3][rl] = o.w;
      }
      // (Lr Z): row rl of the tile, columns cq..cq+3
      const bool own = rl < ni && cq < nj;
      const float4 ar = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.roff[rl], sm.nb.rval[rl], sm.nb.rdeg[rl], sm.nb.rf0[rl], own,
                                   Zin, j0 + cq, I.Lr, I.ldz);
      __syncthreads();  // sm.ac complete
      double dz = 0.0, nz = 0.0;
      float4 zn4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (own) {
        const int64_t i = i0 + rl, jj = j0 + cq;
        const int nv = nj - cq;  // valid entries among the 4
        const float4 z4 = __ldcg(reinterpret_cast<const float4*>(Zin + i * I.ldz + jj));
        const float4 y4 = load4(I.Yt + i * I.ldy + jj, I.yvec, nv);
        const float4 s4 = RESIDENT ? rs : load4(I.S + i * I.lds + jj, I.svec, nv);
        float4 sv4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 ar4 = ar, zz = z4, yy = y4, ss = s4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q < nv) {
            const float z = comp(zz, q), y = comp(yy, q), sp = comp(ss, q);
            // S_j = prox(Z_j - lambda grad g(Z_j)), grad g = 2 (g_c Z Lc + g_r Lr Z)
            const float gr = fmaf(I.two_gr, comp(ar4, q), I.two_gc * sm.ac[rl][cq + q]);
            const float v = fmaf(-lam, gr, z);
            const float dl = v - y;
            const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
            // Z_{j+1} = S_j + ((t_j - 1) / t_{j+1}) (S_j - S_{j-1})
            const float zn = fmaf(mu, sv - sp, sv);
            comp(sv4, q) = sv;
            comp(zn4, q) = zn;
            if (stats) {
              const double d = double(zn) - double(z);
              dz += d * d;
              nz += double(z) * double(z);
            }
          }
        }
        if (a.prev_out && j == a.J) store4(a.prev_out + i * I.lds + jj, s4, a.pvec, nv);  // S_{J-1}
        if (RESIDENT) rs = sv4;
        else store4(I.S + i * I.lds + jj, sv4, I.svec, nv);
        // the padding columns of the last vector get zeros
        *reinterpret_cast<float4*>(Zout + i * I.ldz + jj) = zn4;
      }
      sm.zt[rl][cq] = zn4.x;
      sm.zt[rl][cq + 1] = zn4.y;
      sm.zt[rl][cq + 2] = zn4.z;
      sm.zt[rl][cq + 3] = zn4.w;
      __syncthreads();  // sm.zt complete
      // transposed store: column rl of the tile, rows cq..cq+3
      if (rl < nj && cq < ni) {
        const float4 v = make_float4(sm.zt[cq][rl], sm.zt[cq + 1][rl], sm.zt[cq + 2][rl], sm.zt[cq + 3][rl]);
        *reinterpret_cast<float4*>(ZTout + int64_t(j0 + rl) * I.ldzt + i0 + cq) = v;
      }
      if (stats) {
        dz = block_sum(dz, red);
        nz = block_sum(nz, red);
        if (threadIdx.x == 0) {
          double* st = I.stats + 2 * (j & 3);
          atomicAdd(st, dz);
          atomicAdd(st + 1, nz);
        }
      }
      if (!RESIDENT) __syncthreads();  // before the next tile reuses shared memory
    }
    if (!grid_sync(a.bar)) return;
  }
  if (RESIDENT && blockIdx.x < a.ntiles) {
    const FistaInst& I = a.in[rinst];
    if (rl < rni && cq < rnj) store4(I.S + int64_t(ri0 + rl) * I.lds + rj0 + cq, rs, I.svec, rnj - cq);
  }
  // instances still running at the end did all their iterations
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < a.ninst; i += blockDim.x)
      if (__ldcg(a.in[i].done) == 0) a.in[i].done[1] = jlast;
}

// Z_1 = S_0 = Y~ (Algorithm 1) and the transposed copy of Z_1, one tile per
// block over the batch tile list; the padding of Z's and ZT's rows is zeroed.
// Warm start (a.warm_prev set): S = S_{j0} is kept and Z_{j0+1} =
// S_{j0} + mu_{j0} (S_{j0} - S_{j0-1}), the same operation the iteration
// applies.
__global__ void __launch_bounds__(256) init_batch_kernel(const __grid_constant__ FistaBatchArgs a) {
  __shared__ float tile[TB][TB + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int tl = blockIdx.x; tl < a.ntiles; tl += gridDim.x) {
    const FistaInst& I = a.in[find_inst(a, tl)];
    const int lt = tl - I.tile0;
    const int i0 = (lt / I.ntj) * TB, j0 = (lt % I.ntj) * TB;
    const int ni = min(TB, I.rr - i0), nj = min(TB, I.rc - j0);
    for (int r = warp; r < TB; r += 8) {
      const int64_t i = i0 + r, jj = j0 + lane;
      float y = 0.f;
      if (r < ni && lane < nj) {
        if (a.warm_prev) {
          const float sv = I.S[i * I.lds + jj], sp = a.warm_prev[i * I.lds + jj];
          y = fmaf(a.mu0, sv - sp, sv);
        } else {
          y = I.Yt[i * I.ldy + jj];
          I.S[i * I.lds + jj] = y;
        }
      }
      if (r < ni && jj < I.ldz) {
        I.Z[0][i * I.ldz + jj] = y;
        I.Z[1][i * I.ldz + jj] = 0.f;
      }
      tile[r][lane] = y;
    }
    __syncthreads();
    for (int c = warp; c < TB; c += 8)
      if (c < nj && i0 + lane < I.ldzt) {
        I.ZT[0][int64_t(j0 + c) * I.ldzt + i0 + lane] = tile[lane][c];
        I.ZT[1][int64_t(j0 + c) * I.ldzt + i0 + lane] = 0.f;
      }
    __syncthreads();
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

// ------------------------------------------------ FISTA with dense graphs --
// When both Laplacians are dense (the Kron-reduced graphs of Sec. IV-A), the
// products L_r Z and Z L_c are dense contractions, not gathers. One launch
// per iteration: a block computes a DBM x DBN tile of
//   g = gamma_r (L_r Z_j) + gamma_c (Z_j L_c)
// in FP32 (both products into one accumulator, k-tiles of DBK staged through
// shared memory, the next k-tile prefetched into registers while the current
// one is used), then applies the iteration's update to its entries:
// S_j = prox(Z_j - lambda 2 g), Z_{j+1} = S_j + mu_j (S_j - S_{j-1}).
// Z_j is read from one buffer and Z_{j+1} written to the other, so launches
// order the iterations and no grid barrier is needed.
constexpr int DBM = 32, DBN = 32, DBK = 32, DTHREADS = 64;
constexpr int NRA = DBM * DBK / (4 * DTHREADS), NRB = DBK * DBN / (4 * DTHREADS);  // staged vectors per thread
static_assert(NRA * 4 * DTHREADS == DBM * DBK && NRB * 4 * DTHREADS == DBK * DBN, "whole staging rounds");
static_assert((DBM / 4) * (DBN / 4) == DTHREADS, "one 4 x 4 block of outputs per thread");

struct DenseFistaArgs {
  const float* Lr;  // rr x rr, leading dimension rr
  const float* Lc;  // rc x rc, leading dimension rc
  const float* Zin;
  float* Zout;
  int64_t ldz;
  const float* Yt;
  int64_t ldy;
  float* S;  // S_{j-1} in, S_j out
  int64_t lds;
  const double* lam;
  double* stats;  // the iteration's |Z_{j+1} - Z_j|^2, |Z_j|^2 (added), or null
  int* done;      // done[1] = J on the last iteration, or null
  float* prev_out;  // S_{j-1} (ld lds) on the last iteration, or null
  int J;
  float gr, gc;
  float mu;
  int rr, rc;
  int tiles_r, tiles_c;  // k-tiles of the first (K = rr) and second (K = rc) product
  int vec_lr, vec_lc;    // rows of Lr / Lc allow 16-byte loads (Z's always do)
};

// k-tile t of the concatenated K loop: the A (DBM x DBK) and B (DBK x DBN)
// values this thread stages, zero outside the matrices. Whole 16-byte
// vectors where the rows allow them and the tile lies inside the matrix:
// A vector u covers row (e / 8), columns 4 (e % 8) .. + 3 of the tile, with
// e = threadIdx.x + u DTHREADS (B likewise); otherwise the same elements one
// by one.
__device__ __forceinline__ void dense_fetch(const DenseFistaArgs& a, int t, int i0, int j0, float4 ra[NRA],
                                            float4 rb[NRB]) {
  const bool first = t < a.tiles_r;
  const int k0 = (first ? t : t - a.tiles_r) * DBK;
  const int K = first ? a.rr : a.rc;
  const float* A = first ? a.Lr : a.Zin;
  const int64_t lda = first ? int64_t(a.rr) : a.ldz;
  const float* B = first ? a.Zin : a.Lc;
  const int64_t ldb = first ? a.ldz : int64_t(a.rc);
  const float scale = first ? a.gr : a.gc;
  const bool ka = k0 + DBK <= K;
  const bool va = ka && (first ? a.vec_lr != 0 : true);
  const bool vb = ka && j0 + DBN <= a.rc && (first ? true : a.vec_lc != 0);
#pragma unroll
  for (int u = 0; u < NRA; ++u) {
    const int e = threadIdx.x + u * DTHREADS;
    const int gi = i0 + e / 8, gk = k0 + 4 * (e % 8);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gi < a.rr) {
      const float* p = A + int64_t(gi) * lda + gk;
      if (va) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (gk < K) v.x = __ldg(p);
        if (gk + 1 < K) v.y = __ldg(p + 1);
        if (gk + 2 < K) v.z = __ldg(p + 2);
        if (gk + 3 < K) v.w = __ldg(p + 3);
      }
    }
    ra[u] = make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale);
  }
#pragma unroll
  for (int u = 0; u < NRB; ++u) {
    const int e = threadIdx.x + u * DTHREADS;
    const int gk = k0 + e / 8, gj = j0 + 4 * (e % 8);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gk < K) {
      const float* p = B + int64_t(gk) * ldb + gj;
      if (vb) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (gj < a.rc) v.x = __ldg(p);
        if (gj + 1 < a.rc) v.y = __ldg(p + 1);
        if (gj + 2 < a.rc) v.z = __ldg(p + 2);
        if (gj + 3 < a.rc) v.w = __ldg(p + 3);
      }
    }
    rb[u] = v;
  }
}

__global__ void __launch_bounds__(DTHREADS) fista_dense_kernel(const __grid_constant__ DenseFistaArgs a) {
  __shared__ __align__(16) float As[DBK][DBM + 4];  // As[k][m]
  __shared__ __align__(16) float Bs[DBK][DBN + 4];  // Bs[k][n]
  __shared__ double red[2][DTHREADS / 32];
  const int tx = threadIdx.x % (DBN / 4), ty = threadIdx.x / (DBN / 4);  // 4 columns, 4 rows each
  const int i0 = blockIdx.y * DBM, j0 = blockIdx.x * DBN;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  const int T = a.tiles_r + a.tiles_c;
  float4 ra[NRA], rb[NRB];
  if (T > 0) dense_fetch(a, 0, i0, j0, ra, rb);
  for (int t = 0; t < T; ++t) {
#pragma unroll
    for (int u = 0; u < NRA; ++u) {
      const int e = threadIdx.x + u * DTHREADS, m = e / 8, kq = 4 * (e % 8);
      As[kq][m] = ra[u].x;
      As[kq + 1][m] = ra[u].y;
      As[kq + 2][m] = ra[u].z;
      As[kq + 3][m] = ra[u].w;
    }
#pragma unroll
    for (int u = 0; u < NRB; ++u) {
      const int e = threadIdx.x + u * DTHREADS;
      *reinterpret_cast<float4*>(&Bs[e / 8][4 * (e % 8)]) = rb[u];
    }
    __syncthreads();
    if (t + 1 < T) dense_fetch(a, t + 1, i0, j0, ra, rb);
#pragma unroll 8
    for (int k = 0; k < DBK; ++k) {
      const float4 av = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float am[4] = {av.x, av.y, av.z, av.w}, bn[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(am[r], bn[c], acc[r][c]);
    }
    __syncthreads();
  }
  const float lam = float(*a.lam);
  double dz = 0.0, nz = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= a.rr) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= a.rc) continue;
      const float z = a.Zin[int64_t(i) * a.ldz + j];
      const float y = a.Yt[int64_t(i) * a.ldy + j];
      const float sp = a.S[int64_t(i) * a.lds + j];
      const float v = fmaf(-lam, 2.f * acc[r][c], z);
      const float dl = v - y;
      const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
      const float zn = fmaf(a.mu, sv - sp, sv);
      if (a.prev_out) a.prev_out[int64_t(i) * a.lds + j] = sp;
      a.S[int64_t(i) * a.lds + j] = sv;
      a.Zout[int64_t(i) * a.ldz + j] = zn;
      const double d = double(zn) - double(z);
      dz += d * d;
      nz += double(z) * double(z);
    }
  }
  if (a.stats) {
    dz = warp_sum(dz);
    nz = warp_sum(nz);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[0][w] = dz;
      red[1][w] = nz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sd = 0.0, sn = 0.0;
      for (int q = 0; q < DTHREADS / 32; ++q) {
        sd += red[0][q];
        sn += red[1][q];
      }
      atomicAdd(a.stats, sd);
      atomicAdd(a.stats + 1, sn);
    }
  }
  if (a.done && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) a.done[1] = a.J;
}

// flag[0] |= 1 unless the CSR stores every entry of its n x n matrix in
// row-major order (row pointers i n, columns 0..n-1 in every row).
__global__ void dense_pattern_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int n,
                                     int* __restrict__ flag) {
  const int64_t total = int64_t(n) * n;
  const int64_t g0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x, gs = int64_t(gridDim.x) * blockDim.x;
  bool bad = false;
  for (int64_t t = g0; t < total; t += gs) bad |= col[t] != int32_t(t % n);
  for (int64_t t = g0; t <= n; t += gs) bad |= rowptr[t] != t * n;
  if (bad) atomicOr(flag, 1);
}

}  // namespace

int coop_blocks(const void* kernel, int threads, size_t smem, int want) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  return std::max(1, std::min(want, std::max(occ, 1) * num_sms()));
}

namespace {

int tiles_of(int rr, int rc) { return int(ceil_div(rr, TB) * int64_t(ceil_div(rc, TB))); }

// autotuner cache: launch width chosen for a tile count
std::mutex g_tune_mu;
std::map<int64_t, int> g_tune_cache;

// kernel-parameter tables (large: kept off the stack; one solve at a time
// per table)
std::mutex g_tab_mu;
PowerBatchArgs g_pa;
FistaBatchArgs g_fa;

}  // namespace

// ---------------------------------------------------------------- layout --
InstWs inst_layout(Carve& c, int rr, int rc, size_t zcols) {
  InstWs w{};
  const size_t ldz = size_t(rc + 3) / 4 * 4, ldzt = size_t(rr + 3) / 4 * 4;
  const size_t zc = std::max(ldz, zcols);
  w.Z0 = c.take<float>(size_t(rr) * zc);
  w.Z1 = c.take<float>(size_t(rr) * zc);
  w.ZT0 = c.take<float>(size_t(rc) * ldzt);
  w.ZT1 = c.take<float>(size_t(rc) * ldzt);
  w.scal = c.take<double>(4);
  w.stats = c.take<double>(8);
  w.done = c.take<int>(2);
  return w;
}

BatchWs batch_layout(void* ws, const int* rr, const int* rc, int n) {
  Carve c(ws);
  BatchWs w{};
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.part = c.take<double>(kObjBlocks);
  w.obj = c.take<double>(1);
  {
    std::vector<int> ns(2 * size_t(n));
    for (int i = 0; i < n; ++i) {
      ns[2 * i] = rr[i];
      ns[2 * i + 1] = rc[i];
    }
    w.pscr = c.take<unsigned char>(power_scratch_bytes(ns.data(), 2 * n));
  }
  const bool striped = n == 1 && stripe_candidate(rr[0], rc[0]);
  for (int i = 0; i < n; ++i) w.inst[i] = inst_layout(c, rr[i], rc[i], striped ? stripe_zcols(rc[0]) : 0);
  w.stripe = striped ? stripe_layout(c, rr[0], rc[0]) : StripeWs{};
  w.n = n;
  w.bytes = c.bytes();
  return w;
}

// ----------------------------------------------------------------- solves --
std::mutex g_mu_mu;
bool g_mu_ready[256] = {false};

static cpca_status ensure_mu_table() {
  int dev = 0;
  CPCA_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu_mu);
  if (dev < 0 || dev >= 256 || g_mu_ready[dev]) return CPCA_OK;
  std::vector<float> mu(kMuTable);
  double t = 1.0;
  mu[0] = 0.f;
  for (int j = 1; j < kMuTable; ++j) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    mu[j] = float((t - 1.0) / tn);
    t = tn;
  }
  CPCA_CUDA(cudaMemcpyToSymbol(c_mu, mu.data(), sizeof(float) * kMuTable));
  CPCA_CUDA(cudaMemcpyToSymbol(c_t_last, &t, sizeof(double)));
  g_mu_ready[dev] = true;
  return CPCA_OK;
}

// Warp blocks of a graph list (graph g's first at pa.g[g].w0).
static int assign_warp_blocks(PowerBatchArgs& pa) {
  int nvw = 0;
  for (int g = 0; g < pa.ngraph; ++g) {
    pa.g[g].w0 = nvw;
    nvw += (pa.g[g].L.n + 31) / 32;
  }
  return nvw;
}

size_t power_scratch_bytes(const int* n, int ng) {
  size_t nvw = 0;
  for (int g = 0; g < ng; ++g) nvw += (size_t(n[g]) + 31) / 32;
  return nvw * (2 * 32 * sizeof(float) + 4 * sizeof(double)) + 64;
}

// The power iterations of a graph list: the one-cluster kernels when the
// warp blocks fit (the iterate and the warp sums take a fixed part of the
// opt-in shared memory, the CSR entries the rest), else (forward only) the
// grid-wide kernel on `scratch`. *done = false: reverse asked beyond one
// cluster (nothing launched).
template <int C>
static cudaError_t launch_power_cluster(const PowerBatchArgs& pa, int nvw, int ell_cap, size_t psm,
                                       cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(32 * ((nvw + C - 1) / C));
  cfg.dynamicSmemBytes = psm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nv = nvw, ec = ell_cap;
  void* args[] = {const_cast<PowerBatchArgs*>(&pa), &nv, &ec};
  return cudaLaunchKernelExC(&cfg, (const void*)power_cluster_kernel<C>, args);
}

// Whether a 16-CTA cluster of the forward kernel can run on this device
// (a non-portable cluster size), with the attributes it needs set.
static bool power_cluster16_ok(size_t psm) {
  static std::atomic<int> ok[kMaxDevices];
  return cached_per_device(ok, [&] {
    const void* k = (const void*)power_cluster_kernel<16>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(psm)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = psm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool fits = cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();
    return fits ? 1 : 0;
  }) == 1;
}

static cpca_status power_launch(PowerBatchArgs& pa, bool reverse, void* scratch, cudaStream_t st, bool* done) {
  const int nvw = assign_warp_blocks(pa);
  *done = false;
  const size_t fixed = sizeof(double) * 4 * size_t(nvw) + sizeof(float) * 64 * size_t(nvw);
  const size_t psm = size_t(max_smem_optin());
  const bool c16 = !reverse && nvw > kPowMaxWarps && nvw <= 2 * kPowMaxWarps && fixed < psm / 2 &&
                   power_cluster16_ok(psm);
  if (nvw > kPowMaxWarps && !c16) {
    if (reverse) return CPCA_OK;
    CPCA_CHECK_ARG(scratch, "power iterations: no scratch for %d warp blocks", nvw);
    float* u = static_cast<float*>(scratch);
    double* wq = reinterpret_cast<double*>(u + 2 * 32 * size_t(nvw));
    double* rq = wq + 2 * size_t(nvw);
    const int grid = std::min(2 * num_sms(), coop_blocks((const void*)power_batch_kernel, 512, 0, (nvw + 15) / 16));
    int nv = nvw;
    void* args[] = {&pa, &nv, &u, &wq, &rq};
    CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)power_batch_kernel, dim3(grid), dim3(512), args, 0, st));
    CPCA_LAUNCHED();
    *done = true;
    return CPCA_OK;
  }
  const int ell_cap = int((psm - fixed) / sizeof(int2));
  if (reverse) {
    static PerDeviceOnce attr;
    CPCA_CUDA(once_per_device(attr, [&] {
      return cudaFuncSetAttribute((const void*)power_cluster_reverse_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(psm));
    }));
    power_cluster_reverse_kernel<<<kPowCtas, 32 * ((nvw + kPowCtas - 1) / kPowCtas), psm, st>>>(pa, nvw, ell_cap);
    CPCA_LAUNCHED();
  } else if (c16) {
    CPCA_CUDA(launch_power_cluster<16>(pa, nvw, ell_cap, psm, st));
    CPCA_LAUNCHED();
  } else {
    static PerDeviceOnce attr;
    CPCA_CUDA(once_per_device(attr, [&] {
      return cudaFuncSetAttribute((const void*)power_cluster_kernel<kPowCtas>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(psm));
    }));
    CPCA_CUDA(launch_power_cluster<kPowCtas>(pa, nvw, ell_cap, psm, st));
    CPCA_LAUNCHED();
  }
  *done = true;
  return CPCA_OK;
}

bool power_tape_fits(const CsrView* L, int ng) {
  int nvw = 0;
  for (int g = 0; g < ng; ++g) nvw += (L[g].n + 31) / 32;
  return nvw <= kPowMaxWarps;
}

cpca_status power_tape_run(const PowerTape* P, int ng, int T, uint64_t seed, bool reverse, void* scratch,
                           unsigned int* bar, int* err, cudaStream_t st) {
  CPCA_CHECK_ARG(ng >= 1 && ng <= 2 * kMaxBatch, "power iterations: %d graphs", ng);
  std::unique_ptr<PowerBatchArgs> pa(new PowerBatchArgs{});
  pa->ngraph = ng;
  pa->iters = T;
  pa->seed = seed;
  pa->bar = grid_bar(bar, err);
  for (int g = 0; g < ng; ++g) {
    PowerGraph& G = pa->g[g];
    G.L = P[g].L;
    G.stream = P[g].stream;
    G.out = P[g].rho;
    G.U = P[g].U;
    G.nrm2 = P[g].nrm2;
    G.Ub = P[g].Ub;
    G.rho_bar = P[g].rho_bar;
  }
  if (bar) {
    CPCA_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
    CPCA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  }
  bool done = false;
  CPCA_TRY(power_launch(*pa, reverse, scratch, st, &done));
  CPCA_CHECK_ARG(done, "power iterations: reverse mode needs the rows in one cluster");
  return CPCA_OK;
}

cpca_status fista_batch_run(const BatchProblem* P, int n, int J, double eps, bool want_last,
                            int power_iters, uint64_t power_seed, int blocks, const BatchWs& w,
                            cudaStream_t st, bool dense) {
  CPCA_TRY(ensure_mu_table());
  std::lock_guard<std::mutex> lk(g_tab_mu);
  // the timeout flag covers every launch of this solve (power iterations
  // and FISTA); it is read by read_infos or cpca_frpcag_status
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // power iterations (instances without a given step), then lambda
  PowerBatchArgs& pa = g_pa;
  pa.ngraph = 0;
  for (int i = 0; i < n; ++i) {
    if (P[i].step > 0) continue;
    for (int g = 0; g < 2; ++g) {
      PowerGraph& G = pa.g[pa.ngraph++];
      G = PowerGraph{};
      G.L = g ? P[i].Lc : P[i].Lr;
      G.out = w.inst[i].scal + g;
      G.stream = 2 + g;
    }
  }
  if (pa.ngraph > 0) {
    pa.iters = power_iters;
    pa.seed = power_seed;
    pa.bar = grid_bar(w.bar, w.err);
    CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
    bool done = false;
    CPCA_PROF("power_iter", st);
    CPCA_TRY(power_launch(pa, false, w.pscr, st, &done));
  }
  {
    StepArgs sa{};
    sa.n = n;
    for (int i = 0; i < n; ++i) {
      sa.scal[i] = w.inst[i].scal;
      sa.gamma_r[i] = P[i].gamma_r;
      sa.gamma_c[i] = P[i].gamma_c;
      sa.step[i] = P[i].step;
    }
    step_kernel<<<1, 128, 0, st>>>(sa);
    CPCA_LAUNCHED();
  }
  // FISTA
  FistaBatchArgs& fa = g_fa;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    FistaInst& I = fa.in[i];
    const InstWs& iw = w.inst[i];
    I.Yt = P[i].Yt;
    I.S = P[i].X;
    I.Z[0] = iw.Z0;
    I.Z[1] = iw.Z1;
    I.ZT[0] = iw.ZT0;
    I.ZT[1] = iw.ZT1;
    I.Lr = P[i].Lr;
    I.Lc = P[i].Lc;
    I.lam = iw.scal + 2;
    I.stats = iw.stats;
    I.done = iw.done;
    I.ldy = P[i].ldy;
    I.lds = P[i].ldx;
    I.ldz = (P[i].rc + 3) / 4 * 4;
    I.ldzt = (P[i].rr + 3) / 4 * 4;
    I.yvec = P[i].ldy % 4 == 0 && reinterpret_cast<uintptr_t>(P[i].Yt) % 16 == 0;
    I.svec = P[i].ldx % 4 == 0 && reinterpret_cast<uintptr_t>(P[i].X) % 16 == 0;
    I.two_gr = float(2.0 * P[i].gamma_r);
    I.two_gc = float(2.0 * P[i].gamma_c);
    I.rr = P[i].rr;
    I.rc = P[i].rc;
    I.tile0 = tiles;
    I.ntj = int(ceil_div(P[i].rc, TB));
    tiles += tiles_of(P[i].rr, P[i].rc);
    CPCA_CUDA(cudaMemsetAsync(iw.stats, 0, 8 * sizeof(double), st));
    CPCA_CUDA(cudaMemsetAsync(iw.done, 0, 2 * sizeof(int), st));
  }
  fa.ninst = n;
  fa.ntiles = tiles;
  fa.J = J;
  fa.eps = eps;
  fa.want_last = want_last ? 1 : 0;
  // warm start (single problems only)
  fa.j0 = n == 1 ? P[0].j0 : 0;
  fa.warm_prev = n == 1 && P[0].j0 > 0 ? P[0].warm_prev : nullptr;
  fa.prev_out = n == 1 ? P[0].prev_out : nullptr;
  fa.pvec = fa.prev_out && fa.in[0].svec && reinterpret_cast<uintptr_t>(fa.prev_out) % 16 == 0;
  {
    double t = 1.0, mu = 0.0;  // t_{j0+1} and mu_{j0} by the recurrence of Algorithm 1
    for (int j = 1; j <= fa.j0; ++j) {
      const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
      mu = (t - 1.0) / tn;
      t = tn;
    }
    fa.mu0 = float(mu);
    fa.t0 = t;
  }
  fa.bar = grid_bar(w.bar, w.err);
  // a single problem too large for the resident launch: one striped launch
  // per iteration (no grid barrier; TMA-fed stripes), which sets up its own
  // first iterate
  const size_t smem = sizeof(TileSmem), smem_res = sizeof(TileSmem32);
  const void* kres = (const void*)fista_batch_kernel<true>;
  const void* kstr = (const void*)fista_batch_kernel<false>;
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    const cudaError_t e = cudaFuncSetAttribute(kres, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_res));
    return e != cudaSuccess ? e : cudaFuncSetAttribute(kstr, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  }));
  // 32-bit staged offsets: every instance's Z and ZT below 2^31 entries
  bool small = true;
  for (int i = 0; i < n; ++i)
    small = small && int64_t(P[i].rr) * ((P[i].rc + 3) / 4 * 4) < (int64_t(1) << 31) &&
            int64_t(P[i].rc) * ((P[i].rr + 3) / 4 * 4) < (int64_t(1) << 31);
  const int cap_res = small ? coop_blocks(kres, 256, smem_res, 1 << 30) : 0;
  const int cap_str = coop_blocks(kstr, 256, smem, 1 << 30);
  bool resident = tiles <= cap_res;
  if (n == 1 && J > 0 && !dense && !resident && blocks == 0 && stripe_eligible(P[0].rr, P[0].rc))
    return fista_stripe_run(P[0], w.inst[0], w.stripe, J, eps, want_last, fa.t0, fa.mu0, w.err, st);
  init_batch_kernel<<<std::min(tiles, num_sms() * 8), 256, 0, st>>>(fa);
  CPCA_LAUNCHED();
  if (J == 0) return CPCA_OK;
  if (dense) {  // one instance, both Laplacians dense, fixed J: one launch per iteration
    const BatchProblem& q = P[0];
    const InstWs& iw = w.inst[0];
    DenseFistaArgs da{};
    da.Lr = q.Lr.val;
    da.Lc = q.Lc.val;
    da.ldz = fa.in[0].ldz;
    da.Yt = q.Yt;
    da.ldy = q.ldy;
    da.S = q.X;
    da.lds = q.ldx;
    da.lam = iw.scal + 2;
    da.J = J;
    da.gr = float(q.gamma_r);
    da.gc = float(q.gamma_c);
    da.rr = q.rr;
    da.rc = q.rc;
    da.tiles_r = q.gamma_r != 0 ? int(ceil_div(q.rr, DBK)) : 0;
    da.tiles_c = q.gamma_c != 0 ? int(ceil_div(q.rc, DBK)) : 0;
    da.vec_lr = q.rr % 4 == 0 && reinterpret_cast<uintptr_t>(q.Lr.val) % 16 == 0;
    da.vec_lc = q.rc % 4 == 0 && reinterpret_cast<uintptr_t>(q.Lc.val) % 16 == 0;
    const dim3 grid(ceil_div(q.rc, DBN), ceil_div(q.rr, DBM));
    double t = fa.t0;  // t_{j0+j}; mu as in the constant-memory table
    CPCA_PROF("fista_dense", st);
    for (int j = 1; j <= J; ++j) {
      const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
      da.mu = float((t - 1.0) / tn);
      t = tn;
      da.Zin = fa.in[0].Z[(j - 1) & 1];
      da.Zout = fa.in[0].Z[j & 1];
      da.stats = (j == J && want_last) ? iw.stats + 2 * (J & 3) : nullptr;
      da.done = j == J ? iw.done : nullptr;
      da.prev_out = j == J ? fa.prev_out : nullptr;
      fista_dense_kernel<<<grid, DTHREADS, 0, st>>>(da);
      count_launch();
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        prof_end();
        set_error("dense FISTA launch: %s", cudaGetErrorString(e));
        return CPCA_ERR_CUDA;
      }
    }
    prof_end();
    return CPCA_OK;
  }
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  int grid = resident ? tiles : cap_str;
  if (blocks > 0) {  // explicit launch width (autotuner)
    resident = blocks >= tiles && tiles <= cap_res;
    grid = resident ? tiles : std::min(blocks, cap_str);
  } else if (!resident) {
    std::lock_guard<std::mutex> tl(g_tune_mu);
    auto it = g_tune_cache.find(tiles);
    if (it != g_tune_cache.end()) grid = std::min(it->second, cap_str);
  }
  void* args[] = {&fa};
  CPCA_PROF("fista_persistent", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel(resident ? kres : kstr, dim3(grid), dim3(256), args,
                                        resident ? smem_res : smem, st));
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status fista_objective(const float* Yt, int64_t ldy, int rr, int rc, const CsrView& Lr,
                            const CsrView& Lc, const float* X, int64_t ldx, double gr, double gc,
                            double* part, double* out, cudaStream_t st) {
  CPCA_PROF("fista_objective", st);
  objective_kernel<<<kObjBlocks, 256, 0, st>>>(Yt, ldy, rr, rc, Lr, Lc, X, ldx, gr, gc, part);
  CPCA_LAUNCHED();
  sum_in_order_kernel<<<1, 32, 0, st>>>(part, kObjBlocks, out);
  CPCA_LAUNCHED();
  return CPCA_OK;
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

static cpca_status check_params(const cpca_frpcag_params* prm, const char* who) {
  CPCA_CHECK_ARG(prm, "%s: null params", who);
  CPCA_CHECK_ARG(prm->max_iter >= 0, "%s: max_iter < 0", who);
  CPCA_CHECK_ARG(prm->gamma_r >= 0 && prm->gamma_c >= 0, "%s: negative gamma", who);
  CPCA_CHECK_ARG(prm->eps >= 0, "%s: eps < 0", who);
  CPCA_CHECK_ARG(prm->step > 0 || prm->power_iters >= 1, "%s: power_iters < 1", who);
  CPCA_CHECK_ARG(prm->blocks >= 0, "%s: blocks < 0", who);
  CPCA_CHECK_ARG(prm->start_iter >= 0, "%s: start_iter < 0", who);
  CPCA_CHECK_ARG(prm->start_iter == 0 || prm->start_prev, "%s: start_iter > 0 needs start_prev (S_{j0-1})", who);
  CPCA_CHECK_ARG(!prm->prev_out || prm->eps == 0, "%s: prev_out needs a fixed iteration count (eps = 0)", who);
  return CPCA_OK;
}

static cpca_status read_infos(const BatchProblem* P, int n, const BatchWs& w, int J,
                              cpca_solve_info* const* infos, cudaStream_t st) {
  std::vector<double> hs(size_t(n) * 12);
  std::vector<int> hd(size_t(n) * 2);
  for (int i = 0; i < n; ++i) {
    if (!infos[i]) continue;
    const InstWs& iw = w.inst[i];
    CPCA_TRY(fista_objective(P[i].Yt, P[i].ldy, P[i].rr, P[i].rc, P[i].Lr, P[i].Lc, P[i].X, P[i].ldx,
                             P[i].gamma_r, P[i].gamma_c, w.part, w.obj, st));
    CPCA_CUDA(cudaMemcpyAsync(&hs[size_t(i) * 12], iw.scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&hs[size_t(i) * 12 + 3], iw.stats, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&hs[size_t(i) * 12 + 11], w.obj, sizeof(double), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaMemcpyAsync(&hd[size_t(i) * 2], iw.done, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));  // w.obj is reused per instance
  }
  int err = 0;
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("frpcag: grid barrier timed out");
    return CPCA_ERR_TIMEOUT;
  }
  for (int i = 0; i < n; ++i) {
    if (infos[i] && !std::isfinite(hs[size_t(i) * 12 + 11])) {
      set_error("frpcag: problem %d has a non-finite objective (NaN or Inf in Y~ or the output)", i);
      return CPCA_ERR_NONFINITE;
    }
  }
  for (int i = 0; i < n; ++i) {
    cpca_solve_info* info = infos[i];
    if (!info) continue;
    const double* s = &hs[size_t(i) * 12];
    const int done = J > 0 ? hd[size_t(i) * 2 + 1] : 0;
    const double* last = s + 3 + 2 * (done & 3);
    info->iters = done;
    info->norm_r = s[0];
    info->norm_c = s[1];
    info->step = s[2];
    info->rel_change = done > 0 && last[1] > 0 ? last[0] / last[1] : 0.0;
    info->objective = s[11];
  }
  return CPCA_OK;
}

// Autotuner: time a short run of each candidate launch width and keep the
// fastest (also cached for later solves with the same tile count).
static cpca_status tune_batch(const BatchProblem* P, int n, const BatchWs& w, cudaStream_t st,
                              int* best_blocks, float* best_ms) {
  int tiles = 0;
  for (int i = 0; i < n; ++i) tiles += tiles_of(P[i].rr, P[i].rc);
  const size_t smem = sizeof(TileSmem);
  const int cap_str = coop_blocks((const void*)fista_batch_kernel<false>, 256, smem, 1 << 30);
  const int cap_res = coop_blocks((const void*)fista_batch_kernel<true>, 256, sizeof(TileSmem32), 1 << 30);
  std::vector<int> cands;
  for (int m = 1; m * num_sms() <= cap_str; ++m) cands.push_back(m * num_sms());
  if (cands.empty()) cands.push_back(cap_str);
  if (tiles <= cap_res) cands.push_back(tiles);  // resident
  cudaEvent_t e0, e1;
  CPCA_CUDA(cudaEventCreate(&e0));
  CPCA_CUDA(cudaEventCreate(&e1));
  *best_blocks = 0;
  *best_ms = 1e30f;
  for (int rep = 0; rep < 2; ++rep)
    for (int b : cands) {
      CPCA_CUDA(cudaEventRecord(e0, st));
      CPCA_TRY(fista_batch_run(P, n, 10, 0.0, false, 1, 0, b, w, st));
      CPCA_CUDA(cudaEventRecord(e1, st));
      CPCA_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CPCA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1 && ms < *best_ms) {
        *best_ms = ms;
        *best_blocks = b;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[tiles] = *best_blocks;
  return CPCA_OK;
}

}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_frpcag_workspace_size(int32_t rr, int32_t rc) {
  if (rr <= 0 || rc <= 0) return 0;
  const int a = rr, b = rc;
  return batch_layout(nullptr, &a, &b, 1).bytes;
}

extern "C" cpca_status cpca_frpcag_solve(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                         const cpca_csr* Lr, const cpca_csr* Lc,
                                         const cpca_frpcag_params* prm, float* X, int64_t ldx,
                                         cpca_solve_info* info, void* ws, size_t ws_bytes,
                                         void* stream) {
  clear_error();
  CPCA_RANGE("cpca_frpcag_solve");
  CPCA_CHECK_ARG(Yt && X, "cpca_frpcag_solve: null pointer");
  CPCA_CHECK_ARG(rr > 0 && rc > 0, "cpca_frpcag_solve: empty matrix");
  CPCA_CHECK_ARG(ldyt >= rc && ldx >= rc, "cpca_frpcag_solve: leading dimension too small");
  CPCA_TRY(check_params(prm, "cpca_frpcag_solve"));
  CPCA_TRY(check_csr(Lr, rr, "cpca_frpcag_solve(Lr)"));
  CPCA_TRY(check_csr(Lc, rc, "cpca_frpcag_solve(Lc)"));
  const BatchWs w = batch_layout(ws, &rr, &rc, 1);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_frpcag_solve: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchProblem P{};
  P.Yt = Yt;
  P.ldy = ldyt;
  P.rr = rr;
  P.rc = rc;
  P.Lr = CsrView{Lr->n, Lr->rowptr, Lr->col, Lr->val};
  P.Lc = CsrView{Lc->n, Lc->rowptr, Lc->col, Lc->val};
  P.gamma_r = prm->gamma_r;
  P.gamma_c = prm->gamma_c;
  P.step = prm->step;
  P.X = X;
  P.ldx = ldx;
  P.j0 = prm->start_iter;
  P.warm_prev = prm->start_iter > 0 ? prm->start_prev : nullptr;
  P.prev_out = prm->prev_out;
  // dense Laplacians (every entry stored in row-major order, as the Kron
  // reduction returns them): the products are dense contractions
  bool dense = false;
  if (prm->eps == 0 && prm->blocks == 0 && prm->max_iter > 0 && Lr->nnz == int64_t(rr) * rr &&
      Lc->nnz == int64_t(rc) * rc) {
    int flag = 0;
    CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    dense_pattern_kernel<<<std::min<unsigned>(ceil_div(int64_t(rr) * rr, 256), num_sms() * 8), 256, 0, st>>>(
        Lr->rowptr, Lr->col, rr, w.err);
    CPCA_LAUNCHED();
    dense_pattern_kernel<<<std::min<unsigned>(ceil_div(int64_t(rc) * rc, 256), num_sms() * 8), 256, 0, st>>>(
        Lc->rowptr, Lc->col, rc, w.err);
    CPCA_LAUNCHED();
    CPCA_CUDA(cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));
    CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    dense = flag == 0;
  }
  CPCA_TRY(fista_batch_run(&P, 1, prm->max_iter, prm->eps, info != nullptr, prm->power_iters,
                           prm->power_seed, prm->blocks, w, st, dense));
  if (fault_injected("nan")) CPCA_CUDA(cudaMemsetAsync(X, 0xff, sizeof(float), st));  // a NaN
  if (info) {
    cpca_solve_info* infos[1] = {info};
    CPCA_TRY(read_infos(&P, 1, w, prm->max_iter, infos, st));
  }
  return CPCA_OK;
}

static cpca_status to_problems(const cpca_problem* probs, int32_t count, std::vector<BatchProblem>& P,
                               std::vector<int>& rr, std::vector<int>& rc) {
  CPCA_CHECK_ARG(probs && count >= 1 && count <= kMaxBatch, "batched FISTA: need 1 <= count <= %d",
                 kMaxBatch);
  P.resize(count);
  rr.resize(count);
  rc.resize(count);
  for (int i = 0; i < count; ++i) {
    const cpca_problem& q = probs[i];
    CPCA_CHECK_ARG(q.Yt && q.X && q.rr > 0 && q.rc > 0 && q.ldyt >= q.rc && q.ldx >= q.rc,
                   "batched FISTA: problem %d has bad sizes or pointers", i);
    CPCA_CHECK_ARG(q.gamma_r >= 0 && q.gamma_c >= 0, "batched FISTA: problem %d has negative gamma", i);
    CPCA_TRY(check_csr(&q.Lr, q.rr, "batched FISTA (Lr)"));
    CPCA_TRY(check_csr(&q.Lc, q.rc, "batched FISTA (Lc)"));
    BatchProblem& p = P[i];
    p.Yt = q.Yt;
    p.ldy = q.ldyt;
    p.rr = q.rr;
    p.rc = q.rc;
    p.Lr = CsrView{q.Lr.n, q.Lr.rowptr, q.Lr.col, q.Lr.val};
    p.Lc = CsrView{q.Lc.n, q.Lc.rowptr, q.Lc.col, q.Lc.val};
    p.gamma_r = q.gamma_r;
    p.gamma_c = q.gamma_c;
    p.step = q.step;
    p.X = q.X;
    p.ldx = q.ldx;
    rr[i] = q.rr;
    rc[i] = q.rc;
  }
  return CPCA_OK;
}

extern "C" size_t cpca_frpcag_batched_workspace_size(const cpca_problem* probs, int32_t count) {
  if (!probs || count < 1 || count > kMaxBatch) return 0;
  std::vector<int> rr(count), rc(count);
  for (int i = 0; i < count; ++i) {
    if (probs[i].rr <= 0 || probs[i].rc <= 0) return 0;
    rr[i] = probs[i].rr;
    rc[i] = probs[i].rc;
  }
  return batch_layout(nullptr, rr.data(), rc.data(), count).bytes;
}

extern "C" cpca_status cpca_frpcag_solve_batched(const cpca_problem* probs, int32_t count,
                                                 const cpca_frpcag_params* prm,
                                                 cpca_solve_info* infos, void* ws, size_t ws_bytes,
                                                 void* stream) {
  clear_error();
  CPCA_RANGE("cpca_frpcag_solve_batched");
  CPCA_TRY(check_params(prm, "cpca_frpcag_solve_batched"));
  CPCA_CHECK_ARG(prm->start_iter == 0 && !prm->prev_out,
                 "cpca_frpcag_solve_batched: warm starts are for single solves (start_iter = 0, no prev_out)");
  std::vector<BatchProblem> P;
  std::vector<int> rr, rc;
  CPCA_TRY(to_problems(probs, count, P, rr, rc));
  const BatchWs w = batch_layout(ws, rr.data(), rc.data(), count);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_frpcag_solve_batched: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CPCA_TRY(fista_batch_run(P.data(), count, prm->max_iter, prm->eps, infos != nullptr,
                           prm->power_iters, prm->power_seed, prm->blocks, w, st));
  if (infos) {
    std::vector<cpca_solve_info*> ip(count);
    for (int i = 0; i < count; ++i) ip[i] = infos + i;
    CPCA_TRY(read_infos(P.data(), count, w, prm->max_iter, ip.data(), st));
  }
  return CPCA_OK;
}

extern "C" cpca_status cpca_frpcag_tune_batched(const cpca_problem* probs, int32_t count,
                                                int32_t* blocks, float* ms_per_10_iters, void* ws,
                                                size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_CHECK_ARG(blocks, "cpca_frpcag_tune_batched: null output");
  std::vector<BatchProblem> P;
  std::vector<int> rr, rc;
  CPCA_TRY(to_problems(probs, count, P, rr, rc));
  const BatchWs w = batch_layout(ws, rr.data(), rc.data(), count);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_frpcag_tune_batched: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int b = 0;
  float ms = 0.f;
  CPCA_TRY(tune_batch(P.data(), count, w, st, &b, &ms));
  *blocks = b;
  if (ms_per_10_iters) *ms_per_10_iters = ms;
  return CPCA_OK;
}

// ------------------------------------------------------------------------
// Solve without any allocation: the scratch of cpca_frpcag_solve lives in a
// file-scope device array instead of a caller-provided workspace.
namespace {

constexpr size_t kStaticWsBytes = size_t(CPCA_NOALLOC_WS_BYTES);
// Every GPU that loads this library holds this array until the process exits.
__device__ __align__(256) unsigned char g_noalloc_ws[kStaticWsBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {nullptr};  // device address of g_noalloc_ws, per device

// Device address of the array on the current device, looked up once per
// device (in host code the symbol is only a host-side stand-in).
cpca_status noalloc_base(void** out) {
  int dev = 0;
  CPCA_CUDA(cudaGetDevice(&dev));
  CPCA_CHECK_ARG(dev >= 0 && dev < 256, "cpca_frpcag_solve_noalloc: device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || !p) {
      set_error("cpca_frpcag_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return CPCA_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CPCA_OK;
}

}  // namespace

extern "C" cpca_status cpca_frpcag_status(const void* ws, void* stream) {
  clear_error();
  void* base = const_cast<void*>(ws);
  if (!base) CPCA_TRY(noalloc_base(&base));
  // the flag sits at the same place in every FISTA workspace layout
  const int one = 1;
  const BatchWs w = batch_layout(base, &one, &one, 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int err = 0;
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("frpcag: a grid barrier timed out in the last solve on this workspace");
    return CPCA_ERR_TIMEOUT;
  }
  return CPCA_OK;
}

extern "C" cpca_status cpca_frpcag_solve_noalloc(const float* Yt, int32_t rr, int32_t rc,
                                                 int64_t ldyt, const cpca_csr* Lr,
                                                 const cpca_csr* Lc,
                                                 const cpca_frpcag_params* prm, float* X,
                                                 int64_t ldx, cpca_solve_info* info,
                                                 void* stream) {
  clear_error();
  CPCA_RANGE("cpca_frpcag_solve_noalloc");
  CPCA_CHECK_ARG(rr > 0 && rc > 0, "cpca_frpcag_solve_noalloc: empty matrix");
  const size_t need = cpca_frpcag_workspace_size(rr, rc);
  if (need > kStaticWsBytes) {
    set_error("cpca_frpcag_solve_noalloc: a %d x %d problem needs %zu bytes of scratch, more than "
              "the built-in %zu (use cpca_frpcag_solve with a caller workspace)",
              rr, rc, need, kStaticWsBytes);
    return CPCA_ERR_WORKSPACE;
  }
  void* base = nullptr;
  CPCA_TRY(noalloc_base(&base));
  // Every scratch field that must start at zero is cleared by the solve
  // itself (barrier, statistics, stop flags, power-iteration sums); the rest
  // is written before it is read, so stale contents of earlier calls are
  // harmless. Calls that overlap on the GPU share this array and race.
  return cpca_frpcag_solve(Yt, rr, rc, ldyt, Lr, Lc, prm, X, ldx, info, base, kStaticWsBytes, stream);
}
