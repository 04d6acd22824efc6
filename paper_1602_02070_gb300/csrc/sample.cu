// sample.cu - uniform row/column sampling without replacement and the
// gather Y~ = M_r Y M_c (Sec. III, Eq. Mc).
//
// Each index i gets a counter-based SplitMix64 key; Omega is the rho indices
// with the smallest (key, index). One block per side finds the rho-th
// smallest key by an 8-pass radix select (8-bit digits, MSB first) and then
// compacts the selected indices in index order, so Omega comes out sorted.
// Keys are recomputed on the fly (no scratch memory).
#include "common.cuh"

namespace cpca {
namespace {

constexpr int kSelThreads = 1024;

// Exclusive scan of one int per thread over the block; returns the total.
__device__ int block_exscan(int v, int* sh, int* out) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int o = 1; o < blockDim.x; o <<= 1) {
    int t = tid >= o ? sh[tid - o] : 0;
    __syncthreads();
    sh[tid] += t;
    __syncthreads();
  }
  *out = sh[tid] - v;
  const int total = sh[blockDim.x - 1];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kSelThreads)
sample_select_kernel(uint64_t seed, int p, int n, int rho_r, int rho_c,
                     int32_t* __restrict__ omega_r, int32_t* __restrict__ omega_c, int stream0) {
  const int side = blockIdx.x;
  const int N = side == 0 ? p : n;
  const int rho = side == 0 ? rho_r : rho_c;
  int32_t* out = side == 0 ? omega_r : omega_c;
  const uint64_t s0 = stream_state0(seed, stream0 + side);
  const int tid = threadIdx.x;

  __shared__ int hist[256];
  __shared__ unsigned long long sh_prefix;
  __shared__ int sh_rank;
  __shared__ int scan_buf[kSelThreads];

  // Radix select: find T, the key of rank rho-1 (0-based) in ascending order.
  unsigned long long prefix = 0, mask = 0;
  int rank = rho - 1;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int d = tid; d < 256; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) {
      const uint64_t k = splitmix_at(s0, uint64_t(i) + 1);
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1);
    }
    __syncthreads();
    if (tid == 0) {
      int cum = 0, d = 0;
      for (; d < 256; ++d) {
        if (rank < cum + hist[d]) break;
        cum += hist[d];
      }
      sh_rank = rank - cum;
      sh_prefix = prefix | (uint64_t(d) << shift);
    }
    __syncthreads();
    prefix = sh_prefix;
    rank = sh_rank;
    mask |= 0xFFull << shift;
    __syncthreads();
  }
  const uint64_t T = prefix;
  const int eq_needed = rank + 1;  // keys equal to T taken in index order

  // Compaction in index order: each thread owns a contiguous chunk.
  const int chunk = (N + blockDim.x - 1) / blockDim.x;
  const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
  int n_lt = 0, n_eq = 0;
  for (int i = lo; i < hi; ++i) {
    const uint64_t k = splitmix_at(s0, uint64_t(i) + 1);
    n_lt += k < T;
    n_eq += k == T;
  }
  int lt_before, eq_before;
  block_exscan(n_lt, scan_buf, &lt_before);
  block_exscan(n_eq, scan_buf, &eq_before);
  int pos = lt_before + min(eq_before, eq_needed);
  int eq_seen = eq_before;
  for (int i = lo; i < hi; ++i) {
    const uint64_t k = splitmix_at(s0, uint64_t(i) + 1);
    if (k < T) {
      out[pos++] = i;
    } else if (k == T) {
      if (eq_seen < eq_needed) out[pos++] = i;
      ++eq_seen;
    }
  }
}

__global__ void gather_kernel(const float* __restrict__ Y, int64_t ldy,
                              const int32_t* __restrict__ om_r, const int32_t* __restrict__ om_c,
                              int rr, int rc, float* __restrict__ Yt, int64_t ldyt) {
  const int64_t total = int64_t(rr) * rc;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(t / rc), b = int(t % rc);
    Yt[a * ldyt + b] = __ldg(Y + int64_t(om_r[a]) * ldy + om_c[b]);
  }
}

}  // namespace

cpca_status sample_indices(uint64_t seed, int p, int n, int rho_r, int rho_c,
                           int32_t* om_r, int32_t* om_c, cudaStream_t st) {
  CPCA_PROF("sample_select", st);
  sample_select_kernel<<<2, kSelThreads, 0, st>>>(seed, p, n, rho_r, rho_c, om_r, om_c, 0);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status select_indices(uint64_t seed, int N, int rho, int stream, int32_t* out, cudaStream_t st) {
  sample_select_kernel<<<1, kSelThreads, 0, st>>>(seed, N, 0, rho, 0, out, nullptr, stream);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status gather_submatrix(const float* Y, int64_t ldy, const int32_t* om_r,
                             const int32_t* om_c, int rr, int rc, float* Yt, int64_t ldyt,
                             cudaStream_t st) {
  const int64_t total = int64_t(rr) * rc;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(total, 256), int64_t(num_sms()) * 16);
  CPCA_PROF("sample_gather", st);
  gather_kernel<<<blocks, 256, 0, st>>>(Y, ldy, om_r, om_c, rr, rc, Yt, ldyt);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

}  // namespace cpca

extern "C" cpca_status cpca_sample(uint64_t seed, int32_t p, int32_t n, int32_t rho_r,
                                   int32_t rho_c, const float* Y, int64_t ldy,
                                   int32_t* omega_r, int32_t* omega_c, float* Yt,
                                   int64_t ldyt, void* stream) {
  using namespace cpca;
  clear_error();
  CPCA_RANGE("cpca_sample");
  CPCA_CHECK_ARG(p > 0 && n > 0, "cpca_sample: p, n must be positive");
  CPCA_CHECK_ARG(rho_r > 0 && rho_r <= p && rho_c > 0 && rho_c <= n,
                 "cpca_sample: need 0 < rho_r <= p and 0 < rho_c <= n");
  CPCA_CHECK_ARG(omega_r && omega_c, "cpca_sample: omega_r/omega_c must be device pointers");
  CPCA_CHECK_ARG((Y == nullptr) == (Yt == nullptr), "cpca_sample: give both Y and Yt or neither");
  if (Y) {
    CPCA_CHECK_ARG(ldy >= n && ldyt >= rho_c, "cpca_sample: leading dimension too small");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CPCA_TRY(sample_indices(seed, p, n, rho_r, rho_c, omega_r, omega_c, st));
  if (Y) CPCA_TRY(gather_submatrix(Y, ldy, omega_r, omega_c, rho_r, rho_c, Yt, ldyt, st));
  return CPCA_OK;
}
