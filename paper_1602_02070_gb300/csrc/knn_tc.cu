// knn_tc.cu - tensor-core candidate pass for the kNN graph (sm_103a).
//
// For a block of 128 query points and, in turn, every 256-point base tile
// of its split, the dot products q.b are computed on the 5th-generation
// tensor cores (tcgen05.mma, kind::f16, M = 128, N = 256, FP32 accumulate
// in tensor memory) on a half-precision copy of the points scaled by a
// power of two: the 11-bit significand of TF32 at twice its tensor rate and
// half its bytes. The ranking distance |q|^2 + |b|^2 - 2 q.b then feeds a
// per-query list of the M smallest, kept in registers for M = 32 and in
// shared memory for M = 64 (a per-lane bitmask of the values under the
// current threshold limits the sorted insertions to the few that can enter
// the list). These are only candidates: knn.cu re-scores them with the
// exact FP32 squared distance and certifies the result against the error
// bound of knn_tc_err_rel plus the half copy's absolute terms.
//
// Warp roles (8 warps): warp 0 = TMA producer (one lane), warp 1 = tensor
// memory allocator and MMA issuer (one lane), warps 4-7 = epilogue (warp w
// reads TMEM lanes 32 (w % 4) .. +31, i.e. queries 32 (w - 4) .. +31).
// Operands: K-major, 128-byte swizzle, 64 half columns (128 B) per stage;
// a ring of 4 (M = 32) or 3 (M = 64) stages of (A 16 KB + B 32 KB) guarded
// by full/empty mbarriers; two 256-column accumulators in TMEM (512
// columns) so the epilogue of one base tile overlaps the MMAs of the next.
// Above 32768 dimensions (knn_tc_chunk_ksteps) the second buffer instead
// holds a running sum: the MMAs accumulate 4096 dimensions at a time in the
// first, and the epilogue adds each such chunk into the sum before the
// next chunk starts, which bounds the FP32 accumulation error by 4096
// products rather than d. Every mbarrier wait is bounded: on timeout the
// block raises *err, stops, frees its TMEM and returns.
// Clusters of CL = 2 blocks along the queries share every base tile: each
// block loads 256/CL rows of it with a TMA multicast into every block of the
// cluster (the operand tile of this GPU's own memory, read once from L2 for
// CL blocks), and each block's MMA completion releases the stage in every
// block (tcgen05.commit multicast), so a stage is refilled only when all
// blocks of the cluster are done with it.
#include <cuda.h>
#include <cuda_fp16.h>

#include "knn_internal.cuh"
#include "tma.cuh"

namespace cpca {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, kMaxStages = 4;  // BK: halves per 128-byte row
// M = 32 keeps the per-query lists in registers, which leaves shared memory
// for a fourth operand stage; M = 64 keeps them in shared memory (3 stages).
template <int M>
__host__ __device__ constexpr int stages_of() {
  return M == 32 ? 4 : 3;
}
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 512;

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), sm_100-family descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFF);
  d |= uint64_t(1) << 16;           // leading byte offset (unused for swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;   // stride byte offset
  d |= uint64_t(1) << 46;           // descriptor version
  d |= uint64_t(2) << 61;           // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D F32, A and B F16 (both the same
// type), both K-major, M x N.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// release a stage in every block of the cluster named by `mask`
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
// TMA 2-D load delivered to the same offset in every block of `mask`
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define TMEM_LD_X32(taddr, r)                                                                     \
  asm volatile(                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, " \
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, " \
      "%30, %31}, [%32];"                                                                         \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),       \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),   \
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),             \
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),             \
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])              \
      : "r"(taddr)                                                                                \
      : "memory")

#define TMEM_ST_X32(taddr, r)                                                                     \
  asm volatile(                                                                                   \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "     \
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, " \
      "%29, %30, %31, %32};" ::"r"(taddr),                                                        \
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),     \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),           \
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),         \
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),         \
      "r"(r[29]), "r"(r[30]), "r"(r[31])                                                          \
      : "memory")

struct TcShared {
  uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2];
  uint32_t tmem_base;
  int abort;
};

template <int M, int CL>
__global__ void __launch_bounds__(256, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              int N, int d, const float* __restrict__ nrm, const float* __restrict__ hsc, int splits,
              int kch, int32_t* __restrict__ cand_i, float* __restrict__ cand_d, int* __restrict__ err) {
  // mapB boxes are BN / CL rows: this block's share of a base tile
  extern __shared__ __align__(1024) unsigned char raw[];
  // operand stages must be 1024-byte aligned for the 128-byte swizzle
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  constexpr int STAGES = stages_of<M>();
  constexpr bool kRegLists = M == 32;
  unsigned char* stages = base;
  float* stage_d = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES);  // [32][128] chunk values
  float* ld_ = stage_d + 32 * BM;                                          // [M][128] (shared-memory lists)
  int32_t* li = reinterpret_cast<int32_t*>(ld_ + (kRegLists ? 0 : M * BM));  // [M][128]
  TcShared& sh = *reinterpret_cast<TcShared*>(li + (kRegLists ? 0 : M * BM));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = blockIdx.x * BM;
  const int ntiles = (N + BN - 1) / BN;
  const int per = (ntiles + splits - 1) / splits;
  const int t_lo = blockIdx.y * per, t_hi = min(ntiles, t_lo + per);
  const int nt = max(0, t_hi - t_lo);
  const int nk = (d + BK - 1) / BK;
  // Accumulation chunks: with kch > 0 every kch k-steps start a fresh
  // accumulator in TMEM buffer 0 and the epilogue adds it into the running
  // sum in buffer 1 (FP32, round to nearest), so no accumulation inside the
  // tensor core spans more than kch BK products; kch = 0 accumulates the
  // whole d in one buffer and alternates the two buffers between tiles.
  const int kc = kch > 0 ? kch : nk;
  const int nc = kch > 0 ? (nk + kc - 1) / kc : 1;

  const uint32_t crank = CL > 1 ? cluster_rank() : 0u;
  constexpr uint16_t cmask = uint16_t((1u << CL) - 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], CL);  // released by the MMAs of every block of the cluster
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], 4);
    }
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (CL > 1) cluster_barrier();  // every block's barriers exist before any multicast
  tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int* abort = &sh.abort;

  if (warp == 0) {
    if (lane == 0) {  // ---------------------------------------- TMA producer
      int it = 0;
      for (int t = 0; t < nt && !*abort; ++t) {
        const int n0 = (t_lo + t) * BN;
        for (int k = 0; k < nk; ++k, ++it) {
          const int s = it % STAGES, round = it / STAGES;
          if (!mbar_wait(&sh.empty[s], (round & 1) ^ 1, abort)) break;
          mbar_expect_tx(&sh.full[s], STAGE_BYTES);  // A + all CL shares of B
          unsigned char* sa = stages + s * STAGE_BYTES;
          tma_load_2d(sa, &mapA, &sh.full[s], k * BK, q0);
          if (CL > 1)
            tma_load_2d_mc(sa + A_BYTES + crank * (B_BYTES / CL), &mapB, &sh.full[s], k * BK,
                           n0 + int(crank) * (BN / CL), cmask);
          else
            tma_load_2d(sa + A_BYTES, &mapB, &sh.full[s], k * BK, n0);
        }
      }
      // drain: wait for every issued stage to be consumed before leaving
      for (int s = 0; s < STAGES && it > 0; ++s) {
        const int last = it - 1 - s;
        if (last < 0) break;
        if (!mbar_wait(&sh.empty[last % STAGES], (last / STAGES) & 1, abort)) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------ MMA issuer
      constexpr uint32_t idesc = f16_idesc(BM, BN);
      int it = 0, g = 0;  // g: accumulations issued (chunked mode)
      bool ok = true;
      for (int t = 0; t < nt && ok && !*abort; ++t) {
        for (int c = 0; c < nc && ok; ++c, ++g) {
          const int buf = kch > 0 ? 0 : (t & 1), use = kch > 0 ? g : (t >> 1);
          if (!mbar_wait(&sh.acc_empty[buf], (use & 1) ^ 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + uint32_t(buf * BN);
          const int k_lo = c * kc, k_hi = min(nk, k_lo + kc);
          for (int k = k_lo; k < k_hi; ++k, ++it) {
            const int s = it % STAGES, round = it / STAGES;
            if (!mbar_wait(&sh.full[s], round & 1, abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
            const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)  // 16 halves (32 bytes) per MMA
              umma_f16(dt, ad + uint64_t(kk * 2), bd + uint64_t(kk * 2), idesc,
                       (k != k_lo || kk != 0) ? 1u : 0u);
            if (CL > 1)
              umma_commit_mc(&sh.empty[s], cmask);
            else
              umma_commit(&sh.empty[s]);
          }
          if (ok) umma_commit(&sh.acc_full[buf]);
        }
      }
    }
  } else if (warp >= 4) {  // ------------------------------------- epilogue
    // Ranking value b2 - 2 q.b (|q|^2 is the same for the whole row and is
    // added when the list is written out). Per 32-column chunk every lane
    // builds a bitmask of the values below its current threshold; only
    // those are inserted into its sorted list, so lanes rarely diverge.
    const int ql = (warp - 4) * 32 + lane;  // query within the block = TMEM lane
    const int q = q0 + ql;
    // the lane's list, ascending (equal values keep the earlier index):
    // registers for M = 32 (statically unrolled insertion), else shared memory
    float rd[kRegLists ? M : 1];
    int ri[kRegLists ? M : 1];
    if (kRegLists) {
#pragma unroll
      for (int m = 0; m < (kRegLists ? M : 1); ++m) {
        rd[m] = __int_as_float(0x7f800000);
        ri[m] = -1;
      }
    } else {
      for (int m = 0; m < M; ++m) {
        ld_[m * BM + ql] = __int_as_float(0x7f800000);
        li[m * BM + ql] = -1;
      }
    }
    float thr = __int_as_float(0x7f800000);
    const float m2 = -2.f * hsc[1];  // -2 / s^2: products of the scaled copy back in data units
    const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
    int g = 0;  // accumulations drained (chunked mode)
    for (int t = 0; t < nt; ++t) {
      int buf;
      if (kch > 0) {
        // drain every chunk of this tile into the running sum (buffer 1),
        // then rank from the sum; the MMAs of the next chunk wait only for
        // the drain, so the ranking below overlaps the next tile's first
        // chunk
        bool ok = true;
        for (int c = 0; c < nc; ++c, ++g) {
          if (!mbar_wait(&sh.acc_full[0], g & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll 1
          for (int ch = 0; ch < BN / 32; ++ch) {
            uint32_t a[32], r[32];
            TMEM_LD_X32(tmem + lane_base + uint32_t(ch * 32), a);
            if (c > 0) {
              TMEM_LD_X32(tmem + lane_base + uint32_t(BN + ch * 32), r);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
              for (int i = 0; i < 32; ++i) a[i] = __float_as_uint(__uint_as_float(r[i]) + __uint_as_float(a[i]));
            } else {
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            TMEM_ST_X32(tmem + lane_base + uint32_t(BN + ch * 32), a);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.acc_empty[0]);
        }
        if (!ok) break;
        buf = 1;
      } else {
        buf = t & 1;
        if (!mbar_wait(&sh.acc_full[buf], (t >> 1) & 1, abort)) break;
        tc_fence_after();
      }
      const int n0 = (t_lo + t) * BN;
#pragma unroll 1
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t r[32];
        TMEM_LD_X32(tmem + lane_base + uint32_t(buf * BN + ch * 32), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int nb0 = n0 + ch * 32;
        const float nbl = nb0 + lane < N ? __ldg(nrm + nb0 + lane) : __int_as_float(0x7f800000);
        uint32_t mask = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float dd = fmaf(m2, __uint_as_float(r[i]), __shfl_sync(0xffffffffu, nbl, i));
          stage_d[i * BM + ql] = dd;
          mask |= (dd < thr ? 1u : 0u) << i;
        }
        if (q >= nb0 && q < nb0 + 32) mask &= ~(1u << (q - nb0));
        while (mask) {
          const int i = __ffs(mask) - 1;
          mask &= mask - 1;
          const float dd = stage_d[i * BM + ql];
          if (!(dd < thr)) continue;
          const int jn = nb0 + i;
          if (kRegLists) {
            // every entry above dd moves up one place; dd takes the place
            // after the last entry not above it
#pragma unroll
            for (int p = (kRegLists ? M : 1) - 1; p >= 1; --p) {
              const bool up = rd[p - 1] > dd;
              const bool here = !up && rd[p] > dd;
              rd[p] = up ? rd[p - 1] : (here ? dd : rd[p]);
              ri[p] = up ? ri[p - 1] : (here ? jn : ri[p]);
            }
            if (rd[0] > dd) {
              rd[0] = dd;
              ri[0] = jn;
            }
            thr = rd[(kRegLists ? M : 1) - 1];
          } else {
            int pos = M - 1;
            while (pos > 0 && ld_[(pos - 1) * BM + ql] > dd) {
              ld_[pos * BM + ql] = ld_[(pos - 1) * BM + ql];
              li[pos * BM + ql] = li[(pos - 1) * BM + ql];
              --pos;
            }
            ld_[pos * BM + ql] = dd;
            li[pos * BM + ql] = jn;
            thr = ld_[(M - 1) * BM + ql];
          }
        }
      }
      if (kch == 0) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
      }
    }
    if (q < N) {
      const float nq = nrm[q];
      const int64_t o = (int64_t(blockIdx.y) * N + q) * M;
      if (kRegLists) {
#pragma unroll
        for (int m = 0; m < (kRegLists ? M : 1); ++m) {
          cand_i[o + m] = ri[m];
          cand_d[o + m] = rd[m] + nq;
        }
      } else {
        for (int m = 0; m < M; ++m) {
          cand_i[o + m] = li[m * BM + ql];
          cand_d[o + m] = ld_[m * BM + ql] + nq;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // no block leaves while a peer may still write into its shared memory
  // (multicast loads) or arrive on its barriers (multicast commits)
  if (CL > 1) cluster_barrier();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  if (threadIdx.x == 0 && sh.abort) atomicExch(err, 1);
}

bool make_map(CUtensorMap* map, const __half* H, int N, int d, int64_t ldh, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(d), cuuint64_t(N)};
  cuuint64_t strides[1] = {cuuint64_t(ldh) * 2};
  cuuint32_t box[2] = {cuuint32_t(BK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(H), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool device_is_sm10x() {
  static std::atomic<int> major[kMaxDevices], minor[kMaxDevices];
  const int ma = device_attr(cudaDevAttrComputeCapabilityMajor, major, -1);
  const int mi = device_attr(cudaDevAttrComputeCapabilityMinor, minor, -1);
  cudaGetLastError();
  return ma * 10 + mi == 103;
}

}  // namespace

size_t knn_tc_smem(int M) {
  const int stages = M == 32 ? stages_of<32>() : stages_of<64>();
  return 1024 + size_t(stages) * STAGE_BYTES + size_t(32) * BM * 4 + (M == 32 ? 0 : size_t(M) * BM * 8) +
         sizeof(TcShared) + 64;
}

int64_t knn_half_ld(int d) { return (int64_t(d) + 7) / 8 * 8; }

// Above 32768 dimensions the FP32 accumulation term of the bound below
// exceeds four times the half-rounding term; there the products are summed
// in accumulation chunks of 64 k-steps (4096 dimensions), which costs the
// tensor cores a short wait per chunk while the epilogue adds it up.
int knn_tc_chunk_ksteps(int d) { return d > 32768 ? 64 : 0; }

bool knn_tc_supported(int N, int d, int M) {
  return device_is_sm10x() && N >= 64 && d >= 16 && (M == 32 || M == 64) && encode_fn() != nullptr;
}

cpca_status knn_candidates_tc(const __half* H, int N, int d, int64_t ldh, const float* hsc, int M, int S,
                              const float* nrm, int32_t* cand_i, float* cand_d, int* err, bool* done,
                              cudaStream_t st) {
  *done = false;
  // TMA's rules: row stride a multiple of 16 bytes, 16-byte aligned base
  if (!knn_tc_supported(N, d, M) || (ldh % 8) != 0 || (reinterpret_cast<uintptr_t>(H) & 15) != 0)
    return CPCA_OK;
  // clusters of two query tiles share the base tiles once there are enough
  // query tiles to pair (the last pair may hold a tile past N: its A boxes
  // are zero-filled and its epilogue writes nothing)
  const int qtiles = int(ceil_div(N, BM));
  const int CL = qtiles >= 8 ? 2 : 1;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, H, N, d, ldh, BM) || !make_map(&mapB, H, N, d, ldh, BN / CL)) return CPCA_OK;
  const size_t smem = knn_tc_smem(M);
  const void* kern = M == 32 ? (CL == 2 ? (const void*)knn_tc_kernel<32, 2> : (const void*)knn_tc_kernel<32, 1>)
                             : (CL == 2 ? (const void*)knn_tc_kernel<64, 2> : (const void*)knn_tc_kernel<64, 1>);
  static PerDeviceOnce attr[4];
  CPCA_CUDA(once_per_device(attr[(M == 64) * 2 + (CL == 2)], [&] {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  }));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned((qtiles + CL - 1) / CL * CL), unsigned(S));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(CL);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int kch = knn_tc_chunk_ksteps(d);
  void* args[] = {&mapA,   &mapB, &N, &d, const_cast<float**>(&nrm), const_cast<float**>(&hsc), &S, &kch,
                  &cand_i, &cand_d, &err};
  CPCA_PROF("knn_candidates_tc", st);
  CPCA_CUDA(cudaLaunchKernelExC(&cfg, kern, args));
  CPCA_LAUNCHED();
  *done = true;
  return CPCA_OK;
}

// Bound on |ranking distance - exact distance| / (|q|^2 + |b|^2) for the
// half-precision pass: each scaled coordinate is rounded to nearest with a
// relative error <= 2^-11 (11-bit significand), so each product errs by
// <= (2^-10 + 2^-22) |q_i b_i| and |2 q.b| by <= (2^-10 + 2^-22)
// (|q|^2 + |b|^2); plus FP32 accumulation over the terms of one
// accumulation and the FP32 norms, about (terms + 8) roundings of 2^-23
// each (truncation allowed). With accumulation chunks of c products the
// tensor cores accumulate c terms at a time and the epilogue adds the
// ceil(d / c) chunk sums with round to nearest, adding at most
// (chunks - 1) 2^-24 of sum |q_i b_i|: counted here as chunks 2^-23.
// Coordinates that fall among the half subnormals err absolutely instead;
// that part of the bound depends on the data's scale and is added per query
// from half_scale_kernel's terms.
float knn_tc_err_rel(int d) {
  const int kch = knn_tc_chunk_ksteps(d);
  if (kch == 0) return float(0x1.0p-10 + 0x1.0p-22 + (double(d) + 8.0) * 0x1.0p-23);
  const int64_t nk = (int64_t(d) + BK - 1) / BK, chunks = (nk + kch - 1) / kch;
  return float(0x1.0p-10 + 0x1.0p-22 + (double(kch) * BK + 8.0 + double(chunks)) * 0x1.0p-23);
}

}  // namespace cpca
