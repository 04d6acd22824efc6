// order.cu - locality ordering of a graph's nodes (an internal aid of the
// striped FISTA launch; results do not depend on it).
//
// Nodes are grouped by connected component (components in the order of
// their smallest member), within a component by breadth-first level from
// that member, and within a level by index - a level-set ordering in the
// spirit of Cuthill-McKee. Every edge then joins nodes of one component in
// the same or adjacent levels, so nodes that are processed together (the
// columns of neighbouring stripes) gather from a narrow band of the other
// nodes' rows, which stays in L2.
//
//   order_levels_kernel  cooperative: component labels by min-propagation,
//                        then levels by relaxation, each to its fixed point
//                        (the same labels and levels whatever the update
//                        order), one bounded grid barrier per sweep
//   order_sort_kernel    one block: bitonic sort of the keys
//                        (label, level, index) in shared memory; perm and inv
#include "fista_internal.cuh"

namespace cpca {
namespace {

constexpr int kOrderMaxN = 16384;  // keys sorted in one block's shared memory

__global__ void __launch_bounds__(512)
order_levels_kernel(CsrView L, int32_t* __restrict__ label, int32_t* __restrict__ level,
                    unsigned int* __restrict__ changed, GridBar bar) {
  const int n = L.n;
  const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  // change flags: a ring of three per phase; sweep t sets flag t % 3 and
  // zeroes flag (t + 1) % 3, last read before the barrier that ended sweep t - 1
  for (int v = g0; v < n; v += gs) label[v] = v;
  if (g0 < 6) changed[g0] = 0u;
  if (!grid_sync(bar)) return;
  // components: label = smallest index reachable (monotone min-propagation)
  for (int t = 0; t <= n; ++t) {
    unsigned int* cur = changed + (t % 3);
    if (g0 == 0) changed[(t + 1) % 3] = 0u;
    bool ch = false;
    for (int v = g0; v < n; v += gs) {
      int m = label[v];
      for (int64_t e = L.rowptr[v]; e < L.rowptr[v + 1]; ++e) m = min(m, __ldcg(label + L.col[e]));
      if (m < label[v]) {
        atomicMin(label + v, m);
        ch = true;
      }
    }
    if (ch) atomicOr(cur, 1u);
    if (!grid_sync(bar)) return;
    if (__ldcg(cur) == 0u) break;
  }
  // levels: breadth-first distance from the component's smallest member
  for (int v = g0; v < n; v += gs) level[v] = __ldcg(label + v) == v ? 0 : 0x3fffffff;
  if (!grid_sync(bar)) return;
  for (int t = 0; t <= n; ++t) {
    unsigned int* cur = changed + 3 + (t % 3);
    if (g0 == 0) changed[3 + (t + 1) % 3] = 0u;
    bool ch = false;
    for (int v = g0; v < n; v += gs) {
      int m = __ldcg(level + v);
      for (int64_t e = L.rowptr[v]; e < L.rowptr[v + 1]; ++e) m = min(m, __ldcg(level + L.col[e]) + 1);
      if (m < __ldcg(level + v)) {
        atomicMin(level + v, m);
        ch = true;
      }
    }
    if (ch) atomicOr(cur, 1u);
    if (!grid_sync(bar)) return;
    if (__ldcg(cur) == 0u) break;
  }
}

__global__ void __launch_bounds__(1024)
order_sort_kernel(int n, const int32_t* __restrict__ label, const int32_t* __restrict__ level,
                  int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  extern __shared__ unsigned long long keys[];
  int np = 1;
  while (np < n) np <<= 1;
  for (int v = threadIdx.x; v < np; v += blockDim.x)
    keys[v] = v < n ? (static_cast<unsigned long long>(label[v]) << 40) |
                          (static_cast<unsigned long long>(min(level[v], (1 << 20) - 1)) << 20) |
                          static_cast<unsigned long long>(v)
                    : ~0ull;
  __syncthreads();
  for (int k = 2; k <= np; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = keys[i], b = keys[p];
          if ((a > b) == up) {
            keys[i] = b;
            keys[p] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int v = int(keys[t] & 0xFFFFFull);
    perm[t] = v;
    inv[v] = t;
  }
}

}  // namespace

bool order_supported(int n) { return n >= 2 && n <= kOrderMaxN; }

size_t order_scratch_bytes(int n) { return size_t(2) * n * sizeof(int32_t) + 256; }

cpca_status graph_order(const CsrView& L, int32_t* perm, int32_t* inv, void* scratch, unsigned int* bar,
                        int* err, cudaStream_t st) {
  CPCA_CHECK_ARG(order_supported(L.n), "graph ordering: %d nodes outside [2, %d]", L.n, kOrderMaxN);
  int32_t* label = static_cast<int32_t*>(scratch);
  int32_t* level = label + L.n;
  unsigned int* changed = reinterpret_cast<unsigned int*>(level + L.n);
  CPCA_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  GridBar gb = grid_bar(bar, err);
  CsrView Lv = L;
  const int grid = coop_blocks((const void*)order_levels_kernel, 512, 0, int(ceil_div(L.n, 512)));
  void* args[] = {&Lv, &label, &level, &changed, &gb};
  CPCA_PROF("graph_order", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)order_levels_kernel, dim3(grid), dim3(512), args, 0, st));
  CPCA_LAUNCHED();
  int np = 1;
  while (np < L.n) np <<= 1;
  const size_t smem = size_t(np) * sizeof(unsigned long long);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    return cudaFuncSetAttribute(order_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(size_t(kOrderMaxN) * sizeof(unsigned long long)));
  }));
  order_sort_kernel<<<1, 1024, smem, st>>>(L.n, label, level, perm, inv);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

}  // namespace cpca
