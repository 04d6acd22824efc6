// cluster.cu - the clustering decoder (Sec. V-D, Algorithm 3): k-means on
// the columns of X~ (rho_c points in R^{rho_r}) gives one-hot labels C~;
// every column of C is the harmonic extension of C~ on L_c (Lemma 1, the
// decoder's Jacobi PCG); each node takes the label of its row's largest
// entry (ties: the lowest label).
//
// k-means (the paper leaves its start and stop open): Lloyd's iteration from
// the k columns that the sampling generator picks on stream 5 (ascending
// order), nearest centre by squared Euclidean distance (ties: the lowest
// centre), centres the means of their points (an empty cluster keeps its
// centre), until an assignment step changes no label. One cooperative
// launch: per step, an assignment phase (warp per point, distances by direct
// differences, lane-strided then a butterfly, so every lane holds the same
// sum) and an update phase (block per centre and 256 coordinates, points
// added in index order: deterministic), two grid barriers.
#include <algorithm>

#include "fista_internal.cuh"

namespace cpca {
namespace {

constexpr int kKmeansStream = 5;
constexpr int kClusterKmax = 48;

struct KmArgs {
  const float* P;  // rc x rr points (transposed X~)
  int rr, rc, k, max_iter;
  float* cen;      // k x rr centres
  int* lab;        // rc labels (-1 before the first step)
  unsigned int* changed;  // [2] per step parity
  int* steps;
  GridBar bar;
};

__global__ void transpose_kernel(const float* __restrict__ A, int64_t lda, int rows, int cols,
                                 float* __restrict__ B) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y)
    if (r0 + y < rows && c0 + threadIdx.x < cols) t[y][threadIdx.x] = A[int64_t(r0 + y) * lda + c0 + threadIdx.x];
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y)
    if (c0 + y < cols && r0 + threadIdx.x < rows) B[int64_t(c0 + y) * rows + r0 + threadIdx.x] = t[threadIdx.x][y];
}

// centre c = point init[c]
__global__ void init_centres_kernel(const float* __restrict__ P, int rr, int k, const int32_t* __restrict__ init,
                                    float* __restrict__ cen) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < int64_t(k) * rr;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(e / rr), t = int(e % rr);
    cen[e] = P[int64_t(init[c]) * rr + t];
  }
}

__global__ void __launch_bounds__(256) kmeans_kernel(const __grid_constant__ KmArgs a) {
  const int lane = threadIdx.x & 31;
  const int nwt = (gridDim.x * blockDim.x) >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tchunks = (a.rr + 255) / 256;
  int it = 0;
  for (; it < a.max_iter; ++it) {
    // assignment
    for (int j = gw; j < a.rc; j += nwt) {
      const float* x = a.P + int64_t(j) * a.rr;
      float best = 0.f;
      int bc = 0;
      for (int c = 0; c < a.k; ++c) {
        const float* m = a.cen + int64_t(c) * a.rr;
        float d = 0.f;
        for (int t = lane; t < a.rr; t += 32) {
          const float df = x[t] - __ldcg(m + t);
          d = fmaf(df, df, d);
        }
        d = warp_sumf(d);
        if (c == 0 || d < best) {
          best = d;
          bc = c;
        }
      }
      if (lane == 0) {
        if (a.lab[j] != bc) atomicOr(a.changed + (it & 1), 1u);
        a.lab[j] = bc;
      }
    }
    if (!grid_sync(a.bar)) return;
    if (__ldcg(a.changed + (it & 1)) == 0u) break;
    // update: block (c, coordinate chunk), points in index order
    for (int u = blockIdx.x; u < a.k * tchunks; u += gridDim.x) {
      const int c = u / tchunks, t = (u % tchunks) * 256 + threadIdx.x;
      if (t < a.rr) {
        float s = 0.f;
        int cnt = 0;
        for (int j = 0; j < a.rc; ++j)
          if (__ldcg(a.lab + j) == c) {
            s += a.P[int64_t(j) * a.rr + t];
            ++cnt;
          }
        if (cnt > 0) a.cen[int64_t(c) * a.rr + t] = s / float(cnt);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.changed[(it + 1) & 1] = 0u;
    if (!grid_sync(a.bar)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.steps = min(it + 1, a.max_iter);
}

__global__ void onehot_kernel(const int* __restrict__ lab, int rc, int k, float* __restrict__ R) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < int64_t(rc) * k;
       e += int64_t(gridDim.x) * blockDim.x)
    R[e] = lab[e / k] == int(e % k) ? 1.f : 0.f;
}

// label of row i: the column of its largest entry, the lowest on ties
__global__ void argmax_kernel(const float* __restrict__ C, int n, int k, int32_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* r = C + int64_t(i) * k;
    int b = 0;
    float bv = r[0];
    for (int c = 1; c < k; ++c)
      if (r[c] > bv) {
        bv = r[c];
        b = c;
      }
    out[i] = b;
  }
}

struct ClusterWs {
  float *P, *cen, *R, *C;
  int* lab;
  int32_t* init;
  unsigned int* changed;
  int* steps;
  unsigned int* bar;
  int* err;
  void* hws;
  size_t bytes;
};

ClusterWs cluster_layout(void* ws, int rr, int rc, int n, int k, int64_t nnz_c) {
  Carve c(ws);
  ClusterWs w{};
  w.P = c.take<float>(size_t(rc) * rr);
  w.cen = c.take<float>(size_t(k) * rr);
  w.R = c.take<float>(size_t(rc) * k);
  w.C = c.take<float>(size_t(n) * k);
  w.lab = c.take<int>(rc);
  w.init = c.take<int32_t>(k);
  w.changed = c.take<unsigned int>(2);
  w.steps = c.take<int>(1);
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.hws = c.take<unsigned char>(harmonic_ws_bytes(n, rc, k, nnz_c));
  w.bytes = c.bytes();
  return w;
}

}  // namespace
}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_cluster_decode_workspace_size(int32_t rr, int32_t rc, int32_t n, int32_t k,
                                                     int64_t nnz_c) {
  if (rr <= 0 || rc <= 0 || n < rc || k < 1 || k > kClusterKmax || k > rc || nnz_c < 0) return 0;
  return cluster_layout(nullptr, rr, rc, n, k, nnz_c).bytes;
}

extern "C" cpca_status cpca_cluster_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                           const int32_t* omega_c, int32_t n, const cpca_csr* Lc,
                                           const cpca_cluster_params* prm, int32_t* labels, int32_t* labels_t,
                                           float* C, cpca_cluster_info* info, void* ws, size_t ws_bytes,
                                           void* stream) {
  clear_error();
  CPCA_RANGE("cpca_cluster_decode");
  CPCA_CHECK_ARG(Xt && omega_c && Lc && prm && labels, "cpca_cluster_decode: null pointer");
  CPCA_CHECK_ARG(rr > 0 && rc > 0 && n >= rc && ldxt >= rc, "cpca_cluster_decode: bad sizes");
  CPCA_CHECK_ARG(prm->k >= 1 && prm->k <= kClusterKmax && prm->k <= rc,
                 "cpca_cluster_decode: need 1 <= k <= min(48, rc), got %d", prm->k);
  CPCA_CHECK_ARG(prm->kmeans_iters >= 1 && prm->cg_tol > 0, "cpca_cluster_decode: bad parameters");
  CPCA_TRY(check_csr(Lc, n, "cpca_cluster_decode(Lc)"));
  const int k = prm->k;
  const ClusterWs w = cluster_layout(ws, rr, rc, n, k, Lc->nnz);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_cluster_decode: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CPCA_PROF("kmeans", st);
  transpose_kernel<<<dim3(ceil_div(rc, 32), ceil_div(rr, 32)), dim3(32, 8), 0, st>>>(Xt, ldxt, rr, rc, w.P);
  CPCA_LAUNCHED();
  CPCA_TRY(select_indices(prm->seed, rc, k, kKmeansStream, w.init, st));
  init_centres_kernel<<<std::min<unsigned>(ceil_div(int64_t(k) * rr, 256), 1024u), 256, 0, st>>>(w.P, rr, k, w.init,
                                                                                                 w.cen);
  CPCA_LAUNCHED();
  CPCA_CUDA(cudaMemsetAsync(w.lab, 0xff, sizeof(int) * rc, st));
  CPCA_CUDA(cudaMemsetAsync(w.changed, 0, 2 * sizeof(unsigned int), st));
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  KmArgs a{};
  a.P = w.P;
  a.rr = rr;
  a.rc = rc;
  a.k = k;
  a.max_iter = prm->kmeans_iters;
  a.cen = w.cen;
  a.lab = w.lab;
  a.changed = w.changed;
  a.steps = w.steps;
  a.bar = grid_bar(w.bar, w.err);
  const int want = std::max<int>(int(ceil_div(rc, 8)), k * int(ceil_div(rr, 256)));
  const int grid = coop_blocks((const void*)kmeans_kernel, 256, 0, want);
  void* args[] = {&a};
  CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)kmeans_kernel, dim3(grid), dim3(256), args, 0, st));
  CPCA_LAUNCHED();
  onehot_kernel<<<std::min<unsigned>(ceil_div(int64_t(rc) * k, 256), 1024u), 256, 0, st>>>(w.lab, rc, k, w.R);
  CPCA_LAUNCHED();
  if (labels_t) CPCA_CUDA(cudaMemcpyAsync(labels_t, w.lab, sizeof(int) * rc, cudaMemcpyDeviceToDevice, st));
  int err = 0, steps = 0;
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(&steps, w.steps, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("cpca_cluster_decode: k-means grid barrier timed out");
    return CPCA_ERR_TIMEOUT;
  }
  int cg_it = 0;
  double cg_res = 0.0;
  float* Cout = C ? C : w.C;
  const cpca_status hs = harmonic_extend(Lc, omega_c, n, rc, w.R, k, k, prm->cg_tol, prm->cg_max_iter, Cout, k,
                                         &cg_it, &cg_res, w.hws, st);
  if (hs != CPCA_OK && hs != CPCA_ERR_NOT_CONVERGED) return hs;
  argmax_kernel<<<std::min<unsigned>(ceil_div(n, 256), 1024u), 256, 0, st>>>(Cout, n, k, labels);
  CPCA_LAUNCHED();
  if (info) {
    info->kmeans_steps = steps;
    info->cg_iters = cg_it;
    info->cg_res = cg_res;
  }
  return hs;
}
