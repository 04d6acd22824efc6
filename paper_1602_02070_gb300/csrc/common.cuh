// common.cuh - error plumbing, launch accounting, reductions and a bounded
// grid barrier shared by the libcpca translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "../../include/cpca.h"

namespace cpca {

// ---------------------------------------------------------------- errors --
void set_error(const char* fmt, ...);
void clear_error();
extern std::atomic<uint64_t> g_launches;

inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Per-kernel CUDA-event timing (off by default): CPCA_PROF(name, stream)
// before a launch records a start event when profiling is enabled and the
// name matches the filter; CPCA_LAUNCHED() records the matching end event.
void prof_begin(const char* name, cudaStream_t st);
void prof_end();
#define CPCA_PROF(name, st) ::cpca::prof_begin(name, st)

#define CPCA_CHECK_ARG(cond, ...)                          \
  do {                                                     \
    if (!(cond)) {                                         \
      ::cpca::set_error(__VA_ARGS__);                      \
      return CPCA_ERR_INVALID_ARG;                         \
    }                                                      \
  } while (0)

#define CPCA_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::cpca::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,            \
                        cudaGetErrorString(e_));                               \
      return CPCA_ERR_CUDA;                                                    \
    }                                                                          \
  } while (0)

// NVTX range over an entry point (tracing aid: the call's name on a
// profiler's timeline; header-only NVTX, inert without a profiler).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define CPCA_RANGE(name) ::cpca::NvtxRange cpca_range_(name)

// After a launch: count it and surface launch-configuration errors.
#define CPCA_LAUNCHED()                                                        \
  do {                                                                         \
    ::cpca::count_launch();                                                    \
    ::cpca::prof_end();                                                        \
    cudaError_t e_ = cudaGetLastError();                                       \
    if (e_ != cudaSuccess) {                                                   \
      ::cpca::set_error("%s:%d: kernel launch: %s", __FILE__, __LINE__,        \
                        cudaGetErrorString(e_));                               \
      return CPCA_ERR_CUDA;                                                    \
    }                                                                          \
  } while (0)

#define CPCA_TRY(expr)                 \
  do {                                 \
    cpca_status s_ = (expr);           \
    if (s_ != CPCA_OK) return s_;      \
  } while (0)

// ------------------------------------------------------------ workspace --
// Bump allocator over the caller's workspace; every slice 256-byte aligned.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// ------------------------------------------------------ per-device state --
// Kernel attributes and device queries belong to the current device, so
// everything cached here is cached per device ordinal.
constexpr int kMaxDevices = 64;

inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  return dev;
}

// Runs `fn` (returning cudaError_t) until it succeeds once on the current
// device; later calls on that device return cudaSuccess at once.
struct PerDeviceOnce {
  std::mutex mu;
  bool done[kMaxDevices] = {};
};
template <class F>
cudaError_t once_per_device(PerDeviceOnce& o, F&& fn) {
  const int dev = current_device();
  if (dev >= kMaxDevices) return fn();
  std::lock_guard<std::mutex> lk(o.mu);
  if (o.done[dev]) return cudaSuccess;
  const cudaError_t e = fn();
  if (e == cudaSuccess) o.done[dev] = true;
  return e;
}

// A device attribute of the current device, queried once per device.
inline int device_attr(cudaDeviceAttr attr, std::atomic<int>* cache, int fallback) {
  const int dev = current_device();
  if (dev < kMaxDevices) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, attr, dev) != cudaSuccess || v <= 0) v = fallback;
  if (dev < kMaxDevices) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

inline int num_sms() {
  static std::atomic<int> cache[kMaxDevices];
  return device_attr(cudaDevAttrMultiProcessorCount, cache, 1);
}

// largest dynamic shared memory a block may opt into
inline int max_smem_optin() {
  static std::atomic<int> cache[kMaxDevices];
  return device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, cache, 48 * 1024);
}

// A per-device value (>= 0) computed once by fn() on each device.
template <class F>
int cached_per_device(std::atomic<int>* cache, F&& fn) {
  const int dev = current_device();
  if (dev < kMaxDevices) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v - 1;
  }
  const int v = fn();
  if (dev < kMaxDevices) cache[dev].store(v + 1, std::memory_order_relaxed);
  return v;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return static_cast<unsigned>((a + b - 1) / b); }

// ------------------------------------------------------ SplitMix64 keys --
// Outputs of SplitMix64 (Steele, Lea & Flood 2014) addressed by counter:
// output i (i >= 1) of the generator started at state0 is mix(state0 + i*G).
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t stream_state0(uint64_t seed, int stream) {
  return seed ^ (kGolden * uint64_t(stream + 1));
}
__host__ __device__ inline uint64_t splitmix_at(uint64_t state0, uint64_t i1) {
  return mix64(state0 + i1 * kGolden);
}
__host__ __device__ inline double uniform01_at(uint64_t state0, uint64_t i1) {
  return double(splitmix_at(state0, i1) >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------------ reductions --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a double; every thread gets the result. `red` must hold
// blockDim.x/32 doubles. Contains __syncthreads().
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// ---------------------------------------------------------- grid barrier --
// Counting barrier for cooperative launches (all blocks co-resident): one
// arrival counter (atom.add.acq_rel), the last arriver resets it and bumps
// the generation (release) that the others poll (ld.acquire). Every wait is
// bounded: after kBarrierSpinLimit polls the block records a timeout in
// *err and stops waiting; callers then leave their loops.
constexpr long long kBarrierSpinLimit = 1ll << 23;  // ~ 1-2 s with backoff
constexpr int kBarrierCounters = 1;

struct GridBar {
  unsigned int* count;  // zeroed before the launch
  unsigned int* gen;
  int* err;
  long long limit;      // polls before a wait gives up (kBarrierSpinLimit)
};

// The poll limit new launches take (kBarrierSpinLimit unless a test set a
// shorter one with cpca_debug_set_barrier_spin_limit).
long long barrier_spin_limit();
// Host-side fault injection: true when CPCA_FAULT names this kind.
bool fault_injected(const char* kind);
inline GridBar grid_bar(unsigned int* count, int* err) {
  return GridBar{count, count + kBarrierCounters, err, barrier_spin_limit()};
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int r;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void red_add_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(const GridBar& b) {
  __shared__ int grid_ok;  // thread 0's view of the error flag, for the block
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int g = ld_acquire_u32(b.gen);
    __threadfence();  // the block's writes (ordered by __syncthreads) before arrival
    if (atom_add_acq_rel_u32(b.count, 1u) == nb - 1) {
      *b.count = 0;
      red_add_release_u32(b.gen, 1u);
    } else {
      long long spins = 0;
      while (ld_acquire_u32(b.gen) == g) {
        if (*(volatile int*)b.err) break;
        if (++spins > b.limit) {
          atomicExch(b.err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    grid_ok = *(volatile int*)b.err == 0;
  }
  __syncthreads();
  return grid_ok != 0;
}

}  // namespace cpca
