// decode.cu - subspace-upsampling approximate decoder (Sec. V-C, Lemma 1,
// Eq. Uupsample, Algorithm 2).
//
//  1. Leading singular triplets of X~ by block subspace iteration: FP32
//     tall-skinny products with X~ and X~^T, FP64 Gram matrices, a
//     rank-revealing Cholesky-QR (dependent columns are dropped), and a final
//     Rayleigh-Ritz step whose b x b eigenproblem is solved by parallel-order
//     cyclic Jacobi in one block (FP64).
//  2. k from the ratio rule of Algorithm 2.
//  3. Both upsampling problems, all k columns each, in ONE cooperative PCG
//     kernel: per (side, column) alpha/beta in FP64, FP32 vectors, two
//     bounded grid barriers per iteration. L_aa is applied straight from the
//     full CSR by skipping sampled neighbours (pos < 0).
//  4-6. Column normalisation (FP64 norms), Sigma scaling, X = U Sigma V^T.
#include <cooperative_groups.h>

#include "common.cuh"
#include "fista_internal.cuh"

namespace cpca {
namespace {

constexpr int KMAX_LIMIT = 48;
constexpr int BMAX = 64;

// ------------------------------------------------------ subspace iteration --
__global__ void omega_kernel(float* __restrict__ W, int rows, int b, uint64_t seed) {
  const uint64_t s0 = stream_state0(seed, 4);
  const int64_t total = int64_t(rows) * b;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x)
    W[t] = float(uniform01_at(s0, uint64_t(t) + 1) - 0.5);
}

// C = sum over the chunks of P (nchunk x total floats), in chunk order.
__global__ void gemm_tn_reduce(const float* __restrict__ P, int nchunk, int64_t total, float* __restrict__ C) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < nchunk; ++q) s += P[int64_t(q) * total + t];
    C[t] = s;
  }
}

constexpr int kTnChunks = 64;  // row chunks (column slices) of the split skinny products

// C (m x b) = A (m x n, lda) B (n x b, ld b), b <= BB. A block takes 128
// rows of A and one slice of the n columns (gridDim.y slices) in tiles of
// 32 columns: the A tile is copied row-major into shared memory in 16-byte
// pieces and B's tile stored transposed (Bt[c][k]); the next tile's loads
// are issued before the products of the current one. Each thread owns 4
// rows x BB/8 columns of C (columns j 8 + tx, so that the 16-byte reads of
// Bt by the eight lanes of a quarter warp fall in distinct banks; the A
// reads are broadcasts) and reads, per 4 columns of the tile, 4 + BB/8
// 16-byte values for 16 BB/8 FMAs. The sums run over the columns in order
// (deterministic). One slice writes C; several write their partial
// products to P + y m b, added in slice order by gemm_tn_reduce.
constexpr int NN_RB = 128, NN_KT = 32, NN_LD = NN_KT + 4;
template <int BB, bool VEC>
__global__ void __launch_bounds__(256, BB <= 24 ? 3 : 2)
gemm_nn_tall_k(const float* __restrict__ A, int64_t lda, int m, int n, const float* __restrict__ B, int b,
               float* __restrict__ C, int slice) {
  constexpr int CPT = BB / 8;
  __shared__ __align__(16) float As[NN_RB][NN_LD];
  __shared__ __align__(16) float Bt[BB][NN_LD];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int r0 = blockIdx.x * NN_RB;
  const int kbeg = blockIdx.y * slice, kend = min(n, kbeg + slice);
  if (gridDim.y > 1) C += int64_t(blockIdx.y) * m * b;
  float4 pa[4];
  float pb[CPT];
  // tile loads: A rows ty + 32 q, columns 4 tx .. +3; B elements tid + 256 q
  auto load = [&](int k0) {
    const int kn = kend - k0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = r0 + ty + 32 * q, kk = 4 * tx;
      const float* a = A + int64_t(min(row, m - 1)) * lda + k0 + kk;
      if (row < m && VEC && kk + 3 < kn) {
        pa[q] = __ldg(reinterpret_cast<const float4*>(a));
      } else {
        float v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = (row < m && kk + t < kn) ? __ldg(a + t) : 0.f;
        pa[q] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = tid + 256 * q, k = e / BB, c = e % BB;
      pb[q] = (c < b && k < kn) ? __ldg(B + int64_t(k0 + k) * b + c) : 0.f;
    }
  };
  float acc[4][CPT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
  if (kbeg < kend) load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += NN_KT) {
    __syncthreads();  // the previous tile's reads are done
#pragma unroll
    for (int q = 0; q < 4; ++q) *reinterpret_cast<float4*>(&As[ty + 32 * q][4 * tx]) = pa[q];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = tid + 256 * q;
      Bt[e % BB][e / BB] = pb[q];
    }
    __syncthreads();
    if (k0 + NN_KT < kend) load(k0 + NN_KT);
#pragma unroll
    for (int k4 = 0; k4 < NN_KT; k4 += 4) {
      float4 a[4], bv[CPT];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(&As[4 * ty + i][k4]);
#pragma unroll
      for (int j = 0; j < CPT; ++j) bv[j] = *reinterpret_cast<const float4*>(&Bt[8 * j + tx][k4]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          acc[i][j] = fmaf(a[i].x, bv[j].x, acc[i][j]);
          acc[i][j] = fmaf(a[i].y, bv[j].y, acc[i][j]);
          acc[i][j] = fmaf(a[i].z, bv[j].z, acc[i][j]);
          acc[i][j] = fmaf(a[i].w, bv[j].w, acc[i][j]);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + 4 * ty + i;
    if (row >= m) continue;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = 8 * j + tx;
      if (c < b) C[int64_t(row) * b + c] = acc[i][j];
    }
  }
}

// Slices of the n columns for C = A B: about eight blocks per SM over the
// 128-row blocks, each slice at least 256 columns, at most kTnChunks slices.
static int nn_slices(int m, int n) {
  const int rblocks = int(ceil_div(m, NN_RB));
  return std::max(1, std::min({kTnChunks, int(ceil_div(n, 256)), int(ceil_div(8 * num_sms(), rblocks))}));
}

template <int BB>
static void gemm_nn_tall_run(dim3 g, const float* A, int64_t lda, int m, int n, const float* B, int b, float* C,
                             int slice, bool vec, cudaStream_t st) {
  if (vec)
    gemm_nn_tall_k<BB, true><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, slice);
  else
    gemm_nn_tall_k<BB, false><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, slice);
}

// C (m x b) = A B, split over slices of n when A has few rows (scratch:
// skinny_scratch_floats).
static cpca_status nn_tall(const float* A, int64_t lda, int m, int n, const float* B, int b, float* C,
                           float* scratch, cudaStream_t st) {
  const int ns = nn_slices(m, n);
  const int slice = ns == 1 ? n : int(ceil_div(ceil_div(n, ns), NN_KT)) * NN_KT;
  const int nsl = int(ceil_div(n, slice));
  const bool vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  float* out = nsl > 1 ? scratch : C;
  const dim3 g(unsigned(ceil_div(m, NN_RB)), unsigned(nsl));
  if (b <= 16)
    gemm_nn_tall_run<16>(g, A, lda, m, n, B, b, out, slice, vec, st);
  else if (b <= 24)
    gemm_nn_tall_run<24>(g, A, lda, m, n, B, b, out, slice, vec, st);
  else if (b <= 32)
    gemm_nn_tall_run<32>(g, A, lda, m, n, B, b, out, slice, vec, st);
  else
    gemm_nn_tall_run<BMAX>(g, A, lda, m, n, B, b, out, slice, vec, st);
  CPCA_LAUNCHED();
  if (nsl > 1) {
    const int64_t total = int64_t(m) * b;
    gemm_tn_reduce<<<std::min<unsigned>(ceil_div(total, 256), num_sms() * 4), 256, 0, st>>>(scratch, nsl, total,
                                                                                            C);
    CPCA_LAUNCHED();
  }
  return CPCA_OK;
}

// C (n x b) = A^T B with A (m x n, lda), B (m x b, ld b), b <= BB. A block
// takes 128 columns of A (rows of C) and one chunk of A's rows
// (gridDim.y chunks of `chunk` rows, a multiple of 32) in tiles of 32 rows:
// the A tile is copied into shared memory as it lies (each row's 128
// columns, 512 contiguous bytes), B's 32 rows stored transposed (Bt[c][i]),
// the next tile's loads issued before the products of the current one.
// Each thread owns 4 rows x BB/8 columns of C (columns j 8 + tx, as in
// gemm_nn_tall_k) and reads, per 4 rows of the tile, 4 + BB/8 16-byte
// values for 16 BB/8 FMAs; the sums run over the rows in order. With
// gridDim.y > 1 block (x, y) writes its partial product to C + y n b and
// gemm_tn_reduce adds the chunks in order.
constexpr int TN_CB = 128, TN_LD = TN_CB + 4;
template <int BB>
__global__ void __launch_bounds__(256, BB <= 24 ? 3 : 2)
gemm_tn_tall_k(const float* __restrict__ A, int64_t lda, int m, int n, const float* __restrict__ B, int b,
               float* __restrict__ C, int chunk, bool vec) {
  constexpr int CPT = BB / 8;
  __shared__ __align__(16) float As[NN_KT][TN_LD];
  __shared__ __align__(16) float Bt[BB][NN_LD];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int j0 = blockIdx.x * TN_CB;
  const int ibeg = blockIdx.y * chunk, iend = min(m, ibeg + chunk);
  if (gridDim.y > 1) C += int64_t(blockIdx.y) * n * b;
  float4 pa[4];
  float pb[CPT];
  // tile loads: A rows (tid / 32) + 8 q, columns j0 + 4 (tid % 32) .. +3;
  // B elements tid + 256 q
  auto load = [&](int i0) {
    const int rn = iend - i0, jj = 4 * (tid & 31), jn = n - j0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = (tid >> 5) + 8 * q;
      const float* a = A + int64_t(i0 + min(r, rn - 1)) * lda + j0 + jj;
      if (r < rn && vec && jj + 3 < jn) {
        pa[q] = __ldg(reinterpret_cast<const float4*>(a));
      } else {
        float v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = (r < rn && jj + t < jn) ? __ldg(a + t) : 0.f;
        pa[q] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = tid + 256 * q, r = e / BB, c = e % BB;
      pb[q] = (c < b && r < rn) ? __ldg(B + int64_t(i0 + r) * b + c) : 0.f;
    }
  };
  float acc[4][CPT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
  if (ibeg < iend) load(ibeg);
  for (int i0 = ibeg; i0 < iend; i0 += NN_KT) {
    __syncthreads();  // the previous tile's reads are done
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(&As[(tid >> 5) + 8 * q][4 * (tid & 31)]) = pa[q];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int e = tid + 256 * q;
      Bt[e % BB][e / BB] = pb[q];
    }
    __syncthreads();
    if (i0 + NN_KT < iend) load(i0 + NN_KT);
#pragma unroll
    for (int k4 = 0; k4 < NN_KT; k4 += 4) {
      float4 a[4], bv[CPT];
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = *reinterpret_cast<const float4*>(&As[k4 + t][4 * ty]);
#pragma unroll
      for (int j = 0; j < CPT; ++j) bv[j] = *reinterpret_cast<const float4*>(&Bt[8 * j + tx][k4]);
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        acc[0][j] = fmaf(a[0].x, bv[j].x, acc[0][j]);
        acc[1][j] = fmaf(a[0].y, bv[j].x, acc[1][j]);
        acc[2][j] = fmaf(a[0].z, bv[j].x, acc[2][j]);
        acc[3][j] = fmaf(a[0].w, bv[j].x, acc[3][j]);
        acc[0][j] = fmaf(a[1].x, bv[j].y, acc[0][j]);
        acc[1][j] = fmaf(a[1].y, bv[j].y, acc[1][j]);
        acc[2][j] = fmaf(a[1].z, bv[j].y, acc[2][j]);
        acc[3][j] = fmaf(a[1].w, bv[j].y, acc[3][j]);
        acc[0][j] = fmaf(a[2].x, bv[j].z, acc[0][j]);
        acc[1][j] = fmaf(a[2].y, bv[j].z, acc[1][j]);
        acc[2][j] = fmaf(a[2].z, bv[j].z, acc[2][j]);
        acc[3][j] = fmaf(a[2].w, bv[j].z, acc[3][j]);
        acc[0][j] = fmaf(a[3].x, bv[j].w, acc[0][j]);
        acc[1][j] = fmaf(a[3].y, bv[j].w, acc[1][j]);
        acc[2][j] = fmaf(a[3].z, bv[j].w, acc[2][j]);
        acc[3][j] = fmaf(a[3].w, bv[j].w, acc[3][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = j0 + 4 * ty + i;
    if (j >= n) continue;
#pragma unroll
    for (int jj = 0; jj < CPT; ++jj) {
      const int c = 8 * jj + tx;
      if (c < b) C[int64_t(j) * b + c] = acc[i][jj];
    }
  }
}

static void gemm_tn_tall_launch(dim3 g, const float* A, int64_t lda, int m, int n, const float* B, int b, float* C,
                                int chunk, cudaStream_t st) {
  const bool vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  if (b <= 16)
    gemm_tn_tall_k<16><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, chunk, vec);
  else if (b <= 24)
    gemm_tn_tall_k<24><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, chunk, vec);
  else if (b <= 32)
    gemm_tn_tall_k<32><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, chunk, vec);
  else
    gemm_tn_tall_k<BMAX><<<g, 256, 0, st>>>(A, lda, m, n, B, b, C, chunk, vec);
}


// Row chunks of A^T B, at most kTnChunks of at least 64 rows: enough
// blocks for about two per SM, or, when the columns alone give a block per
// SM (a wide matrix streamed from HBM), about eight per SM, so that more
// rows' loads are in flight.
static int tn_chunks(int m, int n) {
  const int cblocks = int(ceil_div(n, TN_CB));
  const int target = (cblocks >= num_sms() ? 8 : 2) * num_sms();
  return std::max(1, std::min({kTnChunks, int(ceil_div(m, 64)), int(ceil_div(target, cblocks))}));
}

// Scratch (floats) of the split skinny products of an m x n matrix with b
// columns on the other side: tn_tall's row chunks (chunks n b) or nn_tall's
// column slices (slices m b).
static size_t skinny_scratch_floats(int m, int n, int b) {
  const int tc = tn_chunks(m, n), ns = nn_slices(m, n);
  const size_t tn = tc > 1 ? size_t(tc) * n * b : 0, nn = ns > 1 ? size_t(ns) * m * b : 0;
  return std::max<size_t>(1, std::max(tn, nn));
}

// C (n x b) = A^T B, split over row chunks when A is tall (scratch:
// skinny_scratch_floats).
static cpca_status tn_tall(const float* A, int64_t lda, int m, int n, const float* B, int b, float* C,
                           float* scratch, cudaStream_t st) {
  const int cblocks = int(ceil_div(n, TN_CB));
  const int chunks = tn_chunks(m, n);
  if (chunks == 1) {
    gemm_tn_tall_launch(dim3(cblocks, 1), A, lda, m, n, B, b, C, m, st);
    CPCA_LAUNCHED();
    return CPCA_OK;
  }
  const int chunk = int(ceil_div(ceil_div(m, chunks), NN_KT)) * NN_KT;
  const int nch = int(ceil_div(m, chunk));
  gemm_tn_tall_launch(dim3(cblocks, nch), A, lda, m, n, B, b, scratch, chunk, st);
  count_launch();
  const int64_t total = int64_t(n) * b;
  gemm_tn_reduce<<<std::min<unsigned>(ceil_div(total, 256), num_sms() * 4), 256, 0, st>>>(scratch, nch,
                                                                                          total, C);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

constexpr int GRAM_ROWS = 64;

// G += Q^T Q (b x b, FP64, zeroed by the caller): each block takes 64 rows,
// sums their products in FP32 and adds the block total to G in FP64.
__global__ void __launch_bounds__(256)
gram_kernel(const float* __restrict__ Q, int m, int b, double* __restrict__ G) {
  __shared__ float Qs[GRAM_ROWS][BMAX + 1];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * GRAM_ROWS;
  for (int e = tid; e < GRAM_ROWS * b; e += blockDim.x) {
    const int i = e / b, c = e % b;
    Qs[i][c] = (i0 + i < m) ? Q[int64_t(i0 + i) * b + c] : 0.f;
  }
  __syncthreads();
  for (int pr = tid; pr < b * b; pr += blockDim.x) {
    const int a = pr / b, c = pr % b;
    if (c < a) continue;
    float s = 0.f;
#pragma unroll 8
    for (int i = 0; i < GRAM_ROWS; ++i) s = fmaf(Qs[i][a], Qs[i][c], s);
    atomicAdd(G + a * b + c, double(s));
    if (c != a) atomicAdd(G + c * b + a, double(s));
  }
}

// Rank-revealing Cholesky G = R^T R (R upper), right-looking, one block:
// step k takes the pivot, scales row k and updates the trailing triangle in
// parallel (FP64; on this GPU an FP64 warp instruction costs many issue
// cycles, so the work is spread over the block instead of chained in one
// warp). A pivot below 1e-10 of its original diagonal marks a dependent
// direction: row k of R becomes e_k and the direction is dropped (dead).
// Outputs R (b x b, row-major), 1 / R_kk and the dead flags.
__global__ void __launch_bounds__(256)
chol_kernel(const double* __restrict__ G, int b, double* __restrict__ R, double* __restrict__ rdiag,
            int* __restrict__ dead) {
  __shared__ double A[BMAX][BMAX + 1];
  __shared__ double g0[BMAX];
  __shared__ double piv;
  __shared__ int dk;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) A[e / b][e % b] = G[e];
  for (int k = threadIdx.x; k < b; k += blockDim.x) g0[k] = G[k * b + k];
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[k][k];
      const bool dd = !(g0[k] > 1e-300) || !(d > 1e-10 * g0[k]);
      dk = dd;
      piv = dd ? 1.0 : sqrt(d);
      dead[k] = dd;
      rdiag[k] = dd ? 0.0 : 1.0 / piv;
    }
    __syncthreads();
    // row k of R
    for (int j = k + 1 + threadIdx.x; j < b; j += blockDim.x) A[k][j] = dk ? 0.0 : A[k][j] / piv;
    if (threadIdx.x == 0) A[k][k] = piv;
    __syncthreads();
    // trailing update A(i, j) -= R(k, i) R(k, j), k < i <= j
    if (!dk) {
      const int n = b - k - 1;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = k + 1 + e / n, j = k + 1 + e % n;
        if (j >= i) A[i][j] -= A[k][i] * A[k][j];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    R[e] = j >= i ? A[i][j] : 0.0;
  }
}

// Qout = Qin R^-1 row by row (Qin, Qout m x b): x R = q by forward
// substitution, one warp per row, lane c owns column c: x_k = (q_k -
// sum_{i<k} x_i R_ik) / R_kk, then x_k is broadcast and the later lanes
// add x_k R_kc. Dead columns come out zero. FP64 sums, FP32 in and out.
__global__ void __launch_bounds__(256)
trsm_rows_kernel(const float* __restrict__ Qin, int m, int b, const double* __restrict__ R,
                 const double* __restrict__ rdiag, const int* __restrict__ dead, float* __restrict__ Qout) {
  __shared__ double Rs[BMAX][BMAX + 1];
  __shared__ double rd[BMAX];
  __shared__ int dd[BMAX];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Rs[e / b][e % b] = R[e];
  for (int k = threadIdx.x; k < b; k += blockDim.x) {
    rd[k] = rdiag[k];
    dd[k] = dead[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < m; row += nw) {
    const float* q = Qin + int64_t(row) * b;
    double x0 = lane < b ? double(q[lane]) : 0.0, x1 = lane + 32 < b ? double(q[lane + 32]) : 0.0;
    for (int k = 0; k < b; ++k) {
      double xk = k < 32 ? __shfl_sync(0xffffffffu, x0, k) : __shfl_sync(0xffffffffu, x1, k - 32);
      xk = dd[k] ? 0.0 : xk * rd[k];
      if (lane == (k & 31)) {
        if (k < 32) x0 = xk;
        else x1 = xk;
      }
      if (lane > k && lane < b) x0 -= xk * Rs[k][lane];
      if (lane + 32 > k && lane + 32 < b) x1 -= xk * Rs[k][lane + 32];
    }
    if (lane < b) Qout[int64_t(row) * b + lane] = float(x0);
    if (lane + 32 < b) Qout[int64_t(row) * b + lane + 32] = float(x1);
  }
}

// Qout (m x bout) = Qin (m x b) M (b x bout), M FP64 in shared memory.
__global__ void __launch_bounds__(256)
apply_small_kernel(const float* __restrict__ Qin, int m, int b, const double* __restrict__ M,
                   int bout, float* __restrict__ Qout, int ldo, const double* __restrict__ colscale) {
  __shared__ double Ms[BMAX * BMAX];
  for (int e = threadIdx.x; e < b * bout; e += blockDim.x) Ms[e] = M[(e / bout) * b + (e % bout)];
  __syncthreads();
  const int64_t total = int64_t(m) * bout;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / bout), c = int(t % bout);
    double s = 0.0;
    for (int k = 0; k < b; ++k) s += double(Qin[int64_t(i) * b + k]) * Ms[k * bout + c];
    if (colscale) s *= colscale[c];
    Qout[int64_t(i) * ldo + c] = float(s);
  }
}

// Cyclic Jacobi (parallel round-robin order) for the symmetric b x b
// Rayleigh-Ritz matrix: FP32 sweeps, then every eigenvalue is re-evaluated
// as the FP64 Rayleigh quotient e^T H e of its FP32 eigenvector (second-order
// accurate). Eigenvalues descending in lam, eigenvectors as columns of E.
__global__ void __launch_bounds__(256)
jacobi_eig_kernel(const double* __restrict__ H, int b, double* __restrict__ E, double* __restrict__ lam) {
  __shared__ float A[BMAX][BMAX + 1];
  __shared__ float V[BMAX][BMAX + 1];
  __shared__ float cs[BMAX];
  __shared__ int pr[BMAX];
  __shared__ double rq[BMAX];
  __shared__ double red[8];
  __shared__ int perm[BMAX];
  const int bp = b + (b & 1);
  const int tid = threadIdx.x;
  for (int e = tid; e < bp * bp; e += blockDim.x) {
    const int i = e / bp, j = e % bp;
    A[i][j] = (i < b && j < b) ? float(H[i * b + j]) : 0.f;
    V[i][j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < bp * bp; e += blockDim.x) {
      const int i = e / bp, j = e % bp;
      const double a = A[i][j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > 1e-14 * tot)) break;
    for (int round = 0; round < bp - 1; ++round) {
      if (tid < bp / 2) {
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (bp - 1); };
        int p = at(tid), q = at(bp - 1 - tid);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, sn = 0.f;
        const float apq = A[p][q];
        if (apq != 0.f) {
          const float tau = (A[q][q] - A[p][p]) / (2.f * apq);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          sn = t * c;
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = sn;
        pr[2 * tid] = p;
        pr[2 * tid + 1] = q;
      }
      __syncthreads();
      for (int e = tid; e < (bp / 2) * bp; e += blockDim.x) {  // rows: J^T A
        const int k = e / bp, j = e % bp;
        const int p = pr[2 * k], q = pr[2 * k + 1];
        const float c = cs[2 * k], sn = cs[2 * k + 1];
        const float apj = A[p][j], aqj = A[q][j];
        A[p][j] = c * apj - sn * aqj;
        A[q][j] = sn * apj + c * aqj;
      }
      __syncthreads();
      for (int e = tid; e < (bp / 2) * bp; e += blockDim.x) {  // columns: (.) J and V J
        const int k = e / bp, i = e % bp;
        const int p = pr[2 * k], q = pr[2 * k + 1];
        const float c = cs[2 * k], sn = cs[2 * k + 1];
        const float aip = A[i][p], aiq = A[i][q];
        A[i][p] = c * aip - sn * aiq;
        A[i][q] = sn * aip + c * aiq;
        const float vip = V[i][p], viq = V[i][q];
        V[i][p] = c * vip - sn * viq;
        V[i][q] = sn * vip + c * viq;
      }
      __syncthreads();
    }
  }
  // FP64 Rayleigh quotients of the (normalised) eigenvectors
  for (int c = tid; c < b; c += blockDim.x) {
    double nn = 0.0, num = 0.0;
    for (int i = 0; i < b; ++i) {
      double hv = 0.0;
      for (int k = 0; k < b; ++k) hv += H[i * b + k] * double(V[k][c]);
      num += double(V[i][c]) * hv;
      nn += double(V[i][c]) * double(V[i][c]);
    }
    rq[c] = nn > 0 ? num / nn : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < b; ++i) perm[i] = i;
    for (int i = 0; i < b; ++i) {
      int best = i;
      for (int j = i + 1; j < b; ++j)
        if (rq[perm[j]] > rq[perm[best]]) best = j;
      const int t = perm[i];
      perm[i] = perm[best];
      perm[best] = t;
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, c = e % b;
    E[i * b + c] = V[i][perm[c]];
  }
  for (int c = tid; c < b; c += blockDim.x) lam[c] = rq[perm[c]];
}

// s~ = sqrt(max(lam, 0)), 1/s~ (0 where s~ = 0), and k.
__global__ void rank_kernel(const double* __restrict__ lam, int b, double ratio, int k_override,
                            double* __restrict__ s, double* __restrict__ sinv, int* __restrict__ k_out) {
  if (threadIdx.x || blockIdx.x) return;
  for (int i = 0; i < b; ++i) {
    s[i] = sqrt(fmax(lam[i], 0.0));
    sinv[i] = s[i] > 0 ? 1.0 / s[i] : 0.0;
  }
  int k = 0;
  if (s[0] > 0)
    for (int i = 0; i < b; ++i) k += (s[i] / s[0] >= ratio);
  *k_out = k_override > 0 ? k_override : k;
}

// ------------------------------------------------------------------- PCG --
struct CgSide {
  int N, rho, m;
  CsrView L;
  const int32_t* omega;  // sampled nodes, ascending
  int32_t* reach;        // [m]: 1 once a path to a sampled node is known
  int64_t* rp;           // [m + 1] reduced L_aa rows (unsampled index space)
  int32_t* rcol;         // unsampled index of each kept neighbour
  float* rval;
  int32_t* pos;          // [N]: >= 0 unsampled index, < 0 -(sampled index + 1)
  int32_t* abar;         // [m]: node of each unsampled index
  float* minv;           // [m]: 1 / L_aa diagonal (Jacobi)
  const float* R;        // rho x ldr: U~ or V~
  int ldr;
  const float* rhs;      // optional m x k right-hand side (replaces -L_ab R)
  float *x, *r, *z, *p0, *p1, *q;  // m x k
};

struct CgArgs {
  CgSide s[2];
  int k;
  double tol;
  int maxit[2];
  GridBar bar;
  double* acc;       // [2 parity][3][2][KMAX]
  double* acc_init;  // [3][2][KMAX]
  int* out_iters;    // [2][KMAX]
  double* out_res;   // [2][KMAX]
  int* status;       // [0]: 1 = PCG breakdown, 2 = a component without samples
  unsigned int* changed;  // [3] reachability round counters
};

__global__ void cg_setup_kernel(CgSide S0, CgSide S1) {
  const CgSide& S = blockIdx.y == 0 ? S0 : S1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.N; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = S.rho;  // lower_bound of i in omega
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (S.omega[mid] < i) lo = mid + 1; else hi = mid;
    }
    if (lo < S.rho && S.omega[lo] == i) {
      S.pos[i] = -(lo + 1);
    } else {
      const int t = i - lo;
      S.pos[i] = t;
      S.abar[t] = i;
      float dg = 0.f;
      for (int64_t e = S.L.rowptr[i]; e < S.L.rowptr[i + 1]; ++e)
        if (S.L.col[e] == i) dg = S.L.val[e];
      S.minv[t] = dg > 0.f ? 1.f / dg : 1.f;
    }
  }
}

// L_aa in its own CSR over the unsampled index space: count, scan, fill.
__global__ void laa_count_kernel(CgSide S0, CgSide S1) {
  const CgSide& S = blockIdx.y == 0 ? S0 : S1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.m; t += gridDim.x * blockDim.x) {
    const int node = S.abar[t];
    int c = 0;
    for (int64_t e = S.L.rowptr[node]; e < S.L.rowptr[node + 1]; ++e) c += S.pos[S.L.col[e]] >= 0;
    S.rp[t + 1] = c;
  }
}
__global__ void laa_scan_kernel(CgSide S0, CgSide S1) {
  const CgSide& S = blockIdx.x == 0 ? S0 : S1;
  __shared__ int64_t sh[1024];
  const int tid = threadIdx.x, nt = blockDim.x, m = S.m;
  const int chunk = (m + nt - 1) / nt;
  const int lo = min(m, tid * chunk), hi = min(m, lo + chunk);
  int64_t sum = 0;
  for (int t = lo; t < hi; ++t) sum += S.rp[t + 1];
  sh[tid] = sum;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const int64_t v = tid >= o ? sh[tid - o] : 0;
    __syncthreads();
    sh[tid] += v;
    __syncthreads();
  }
  // in place: rp[t + 1] = sum of the counts of rows 0..t (each thread only
  // touches rp[lo + 1 .. hi]), rp[0] = 0
  int64_t run = sh[tid] - sum;
  for (int t = lo; t < hi; ++t) {
    run += S.rp[t + 1];
    S.rp[t + 1] = run;
  }
  if (tid == 0) S.rp[0] = 0;
}
__global__ void laa_fill_kernel(CgSide S0, CgSide S1) {
  const CgSide& S = blockIdx.y == 0 ? S0 : S1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.m; t += gridDim.x * blockDim.x) {
    const int node = S.abar[t];
    int64_t w = S.rp[t];
    for (int64_t e = S.L.rowptr[node]; e < S.L.rowptr[node + 1]; ++e) {
      const int ps = S.pos[S.L.col[e]];
      if (ps >= 0) {
        S.rcol[w] = ps;
        S.rval[w] = S.L.val[e];
        ++w;
      }
    }
  }
}

// Per-thread partial dot products -> per (kind, side, column) block sums ->
// one FP64 atomic per block and column into gacc[kind][side][KMAX_LIMIT].
// Thread gtid owns column gtid % k, so the block sum for column c adds the
// threads tid = c - base (mod k), base = (blockIdx.x * blockDim.x) % k.
__device__ __forceinline__ void block_flush(double* shm, const double (*acc)[2], int kind0,
                                            int nkind, int k, double* gacc) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = 0; q < nkind; ++q)
    for (int sd = 0; sd < 2; ++sd) shm[(q * 2 + sd) * nt + tid] = acc[kind0 + q][sd];
  __syncthreads();
  const int base = int((int64_t(blockIdx.x) * nt) % k);
  for (int e = tid; e < nkind * 2 * k; e += nt) {
    const int q = e / (2 * k), sd = (e / k) & 1, c = e % k;
    int t2 = (c - base) % k;
    if (t2 < 0) t2 += k;
    double sum = 0.0;
    for (; t2 < nt; t2 += k) sum += shm[(q * 2 + sd) * nt + t2];
    if (sum != 0.0) atomicAdd(gacc + ((kind0 + q) * 2 + sd) * KMAX_LIMIT + c, sum);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256)
cg_kernel(CgArgs a) {
  __shared__ double shm[3 * 2 * 256];
  __shared__ double rz[2][KMAX_LIMIT], beta[2][KMAX_LIMIT], alpha[2][KMAX_LIMIT], bn[2][KMAX_LIMIT];
  __shared__ double lastrr[2][KMAX_LIMIT];
  __shared__ int active[2][KMAX_LIMIT], iters[2][KMAX_LIMIT];
  __shared__ int any_active;
  __shared__ int blk_changed;
  const int k = a.k;
  const int nacc = 2 * KMAX_LIMIT;
  const int m0 = a.s[0].m;
  const int64_t rows = int64_t(m0) + a.s[1].m;
  const int64_t gstride = int64_t(gridDim.x) * blockDim.x;
  const int64_t gtid = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  // fixed column per thread, rows t0, t0 + tstride, ... over both sides
  const int mycol = int(gtid % k);
  const int64_t tstride = gstride / k;
  const int64_t t0 = gtid / k;
  const bool owns = gtid < tstride * k;

  // Reachability: L_aa is invertible exactly when every connected component
  // of the graph holds a sampled node. Rounds of frontier growth from the
  // sampled set until a round changes nothing (at most m + 1 rounds).
  for (int64_t g = gtid; g < rows; g += gstride) {
    const int sd = g < m0 ? 0 : 1;
    a.s[sd].reach[sd ? g - m0 : g] = 0;
  }
  if (!grid_sync(a.bar)) return;
  for (int round = 0; round <= max(a.s[0].m, a.s[1].m) + 1; ++round) {
    if (threadIdx.x == 0) blk_changed = 0;
    __syncthreads();
    for (int64_t g = gtid; g < rows; g += gstride) {
      const int sd = g < m0 ? 0 : 1;
      const CgSide& S = a.s[sd];
      const int t = int(sd ? g - m0 : g);
      if (__ldcg(S.reach + t)) continue;
      const int node = S.abar[t];
      for (int64_t e = S.L.rowptr[node]; e < S.L.rowptr[node + 1]; ++e) {
        const int j = S.L.col[e];
        if (j == node || S.L.val[e] == 0.f) continue;
        const int ps = S.pos[j];
        if (ps < 0 || __ldcg(S.reach + ps)) {
          S.reach[t] = 1;
          blk_changed = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_changed) atomicAdd(a.changed + round % 3, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.changed[(round + 1) % 3] = 0;
    if (!grid_sync(a.bar)) return;
    if (__ldcg(a.changed + round % 3) == 0) break;
  }
  for (int64_t g = gtid; g < rows; g += gstride) {
    const int sd = g < m0 ? 0 : 1;
    if (!__ldcg(a.s[sd].reach + (sd ? g - m0 : g))) atomicOr(a.status, 2);
  }

  double acc[3][2];
  // r = b = -L_ab R, x = 0, z = M^-1 r, p_prev = 0
  acc[0][0] = acc[0][1] = acc[1][0] = acc[1][1] = acc[2][0] = acc[2][1] = 0.0;
  if (owns)
    for (int64_t tt = t0; tt < rows; tt += tstride) {
      const int sd = tt < m0 ? 0 : 1;
      const CgSide& S = a.s[sd];
      const int t = int(sd ? tt - m0 : tt);
      const int64_t l = int64_t(t) * k + mycol;
      const int node = S.abar[t];
      float bv = 0.f;
      if (S.rhs) {
        bv = S.rhs[l];
      } else {
        for (int64_t e = S.L.rowptr[node]; e < S.L.rowptr[node + 1]; ++e) {
          const int ps = S.pos[S.L.col[e]];
          if (ps < 0) bv = fmaf(-S.L.val[e], S.R[int64_t(-ps - 1) * S.ldr + mycol], bv);
        }
      }
      const float zv = S.minv[t] * bv;
      S.r[l] = bv;
      S.z[l] = zv;
      S.x[l] = 0.f;
      S.p1[l] = 0.f;
      acc[0][sd] += double(bv) * bv;
      acc[1][sd] += double(bv) * zv;
      acc[2][sd] += double(bv) * bv;
    }
  block_flush(shm, acc, 0, 3, k, a.acc_init);
  if (!grid_sync(a.bar)) return;
  for (int e = threadIdx.x; e < 2 * k; e += blockDim.x) {
    const int sd = e / k, c = e % k;
    const double bb = __ldcg(a.acc_init + (0 * 2 + sd) * KMAX_LIMIT + c);
    bn[sd][c] = sqrt(bb);
    rz[sd][c] = __ldcg(a.acc_init + (1 * 2 + sd) * KMAX_LIMIT + c);
    const double rr = __ldcg(a.acc_init + (2 * 2 + sd) * KMAX_LIMIT + c);
    lastrr[sd][c] = rr;
    active[sd][c] = (a.s[sd].m > 0) && (sqrt(rr) > a.tol * bn[sd][c]) && (a.maxit[sd] > 0);
    beta[sd][c] = 0.0;
    iters[sd][c] = 0;
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int any = 0;
      for (int e = 0; e < 2 * k; ++e) any |= active[e / k][e % k];
      any_active = any;
    }
    __syncthreads();
    if (!any_active) break;
    const int par = it & 1;
    double* accp = a.acc + par * 3 * nacc;
    // Phase Q: p = z + beta p_prev (own rows and, on the fly, neighbours);
    // q = L_aa p; accumulate p.q
    acc[0][0] = acc[0][1] = 0.0;
    if (owns)
      for (int64_t tt = t0; tt < rows; tt += tstride) {
        const int sd = tt < m0 ? 0 : 1;
        if (!active[sd][mycol]) continue;
        const CgSide& S = a.s[sd];
        const int t = int(sd ? tt - m0 : tt);
        const int64_t l = int64_t(t) * k + mycol;
        float* pcur = par ? S.p1 : S.p0;
        const float* pprev = par ? S.p0 : S.p1;
        const float bt = float(beta[sd][mycol]);
        const float pv = fmaf(bt, pprev[l], S.z[l]);
        pcur[l] = pv;
        float qv = 0.f;
        const int64_t e1 = S.rp[t + 1];
        int64_t e = S.rp[t];
        // neighbours were written by other blocks in this launch: bypass L1
        for (; e + 4 <= e1; e += 4) {
          float pv4[4], zv4[4], w4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t o = int64_t(S.rcol[e + u]) * k + mycol;
            w4[u] = S.rval[e + u];
            pv4[u] = __ldcg(pprev + o);
            zv4[u] = __ldcg(S.z + o);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) qv = fmaf(w4[u], fmaf(bt, pv4[u], zv4[u]), qv);
        }
        for (; e < e1; ++e) {
          const int64_t o = int64_t(S.rcol[e]) * k + mycol;
          qv = fmaf(S.rval[e], fmaf(bt, __ldcg(pprev + o), __ldcg(S.z + o)), qv);
        }
        S.q[l] = qv;
        acc[0][sd] += double(pv) * qv;
      }
    block_flush(shm, acc, 0, 1, k, accp);
    if (!grid_sync(a.bar)) return;
    for (int e = threadIdx.x; e < 2 * k; e += blockDim.x) {
      const int sd = e / k, c = e % k;
      if (!active[sd][c]) continue;
      const double pq = __ldcg(accp + sd * KMAX_LIMIT + c);
      if (!(pq > 0.0)) {
        alpha[sd][c] = 0.0;
        if (blockIdx.x == 0) atomicOr(a.status, 1);  // L_aa not positive definite
      } else {
        alpha[sd][c] = rz[sd][c] / pq;
      }
    }
    __syncthreads();
    // Phase U: x += alpha p; r -= alpha q; z = M^-1 r; accumulate r.z, r.r
    acc[1][0] = acc[1][1] = acc[2][0] = acc[2][1] = 0.0;
    if (owns)
      for (int64_t tt = t0; tt < rows; tt += tstride) {
        const int sd = tt < m0 ? 0 : 1;
        if (!active[sd][mycol]) continue;
        const CgSide& S = a.s[sd];
        const int t = int(sd ? tt - m0 : tt);
        const int64_t l = int64_t(t) * k + mycol;
        const float* pcur = par ? S.p1 : S.p0;
        const float al = float(alpha[sd][mycol]);
        S.x[l] = fmaf(al, pcur[l], S.x[l]);
        const float rv = fmaf(-al, S.q[l], S.r[l]);
        S.r[l] = rv;
        const float zv = S.minv[t] * rv;
        S.z[l] = zv;
        acc[1][sd] += double(rv) * zv;
        acc[2][sd] += double(rv) * rv;
      }
    block_flush(shm, acc, 1, 2, k, accp);
    if (blockIdx.x == 0) {
      double* other = a.acc + (1 - par) * 3 * nacc;
      for (int e = threadIdx.x; e < 3 * nacc; e += blockDim.x) other[e] = 0.0;
    }
    if (!grid_sync(a.bar)) return;
    for (int e = threadIdx.x; e < 2 * k; e += blockDim.x) {
      const int sd = e / k, c = e % k;
      if (!active[sd][c]) continue;
      const double rzn = __ldcg(accp + (1 * 2 + sd) * KMAX_LIMIT + c);
      const double rr = __ldcg(accp + (2 * 2 + sd) * KMAX_LIMIT + c);
      beta[sd][c] = rz[sd][c] != 0.0 ? rzn / rz[sd][c] : 0.0;
      rz[sd][c] = rzn;
      lastrr[sd][c] = rr;
      iters[sd][c] += 1;
      if (!(sqrt(rr) > a.tol * bn[sd][c]) || iters[sd][c] >= a.maxit[sd] || alpha[sd][c] == 0.0)
        active[sd][c] = 0;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < 2 * k; e += blockDim.x) {
      const int sd = e / k, c = e % k;
      a.out_iters[sd * KMAX_LIMIT + c] = iters[sd][c];
      a.out_res[sd * KMAX_LIMIT + c] = bn[sd][c] > 0 ? sqrt(lastrr[sd][c]) / bn[sd][c] : 0.0;
    }
  }
}

// U (N x ldu): sampled rows from R (U~ or V~), unsampled rows from x.
__global__ void assemble_side_kernel(int N, int k, int ldu, const int32_t* __restrict__ pos,
                                     const float* __restrict__ R, int ldr, const float* __restrict__ x,
                                     float* __restrict__ U) {
  const int64_t total = int64_t(N) * ldu;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / ldu), c = int(t % ldu);
    float v = 0.f;
    if (c < k) {
      const int ps = pos[i];
      v = ps < 0 ? R[int64_t(-ps - 1) * ldr + c] : x[int64_t(ps) * k + c];
    }
    U[t] = v;
  }
}

constexpr int NORM_BLOCKS = 128;

__global__ void colnorm_partial_kernel(const float* __restrict__ U, int N, int k, int ldu,
                                       double* __restrict__ part) {
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(N, lo + per);
  // each thread owns one column and a fixed row stride: deterministic order
  const int c = threadIdx.x % KMAX_LIMIT, lane_row = threadIdx.x / KMAX_LIMIT;
  const int rows_par = blockDim.x / KMAX_LIMIT;
  double acc = 0.0;
  if (c < k && lane_row < rows_par)
    for (int i = lo + lane_row; i < hi; i += rows_par) {
      const double v = U[int64_t(i) * ldu + c];
      acc += v * v;
    }
  __shared__ double tmp[256];
  tmp[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < KMAX_LIMIT) {
    double t = 0.0;
    for (int r = 0; r < rows_par; ++r) t += tmp[r * KMAX_LIMIT + threadIdx.x];
    part[int64_t(blockIdx.x) * KMAX_LIMIT + threadIdx.x] = t;
  }
}

// inv norms for both sides and sigma = scale * s~.
__global__ void norm_finish_kernel(const double* __restrict__ pu, const double* __restrict__ pv,
                                   int nblk, int k, const double* __restrict__ s_tilde, double scale,
                                   double* __restrict__ invu, double* __restrict__ invv,
                                   double* __restrict__ sigma, int ksig) {
  for (int c = threadIdx.x; c < KMAX_LIMIT; c += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblk; ++i) {
      a += pu[int64_t(i) * KMAX_LIMIT + c];
      b += pv[int64_t(i) * KMAX_LIMIT + c];
    }
    invu[c] = (c < k && a > 0) ? 1.0 / sqrt(a) : 0.0;
    invv[c] = (c < k && b > 0) ? 1.0 / sqrt(b) : 0.0;
    if (c < ksig) sigma[c] = c < k ? scale * s_tilde[c] : 0.0;
  }
}

__global__ void scale_cols_kernel(float* __restrict__ U, int64_t total, int ldu, const double* __restrict__ inv) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x)
    U[t] = float(double(U[t]) * inv[t % ldu]);
}

// X (p x n) = U diag(sigma) V^T, X(i, j) = sum_c (U(i, c) sigma_c) V(j, c)
// summed in c order, sigma_c rounded to FP32 (Algorithm 2, step 6; also
// the projections of approximate decoders 2 and 3 with sigma = 1). A block
// owns 256 columns and OUT_RT row tiles of 32 rows: V's 256 x k slice is
// read row by row (consecutive threads take consecutive c) and staged once
// in shared memory, k-major; per row tile the 32 x k slice of U is staged
// the same way, scaled by sigma; each thread then computes an 8 x 4 block
// of X (8 scaled U values and 4 V values per c from shared memory, 32 FMAs
// issued as 16 packed two-lane FMAs on pairs of rows, each lane rounded as
// fmaf) and writes its 8 rows as 16-byte streaming stores. At k = 20 the
// FMAs, 20 per entry, take longer than the 4 B per entry written.
constexpr int OUT_RT = 16, OUT_VLD = 256 + 4, OUT_ULD = 32 + 4;
__global__ void __launch_bounds__(256)
output_kernel(const float* __restrict__ U, int ldu, const float* __restrict__ V, int ldv,
              const double* __restrict__ sigma, int k, int p, int n, float* __restrict__ X, int64_t ldx) {
  extern __shared__ __align__(16) float osm[];
  float* VsT = osm;                 // [k][OUT_VLD]
  float* UsT = osm + k * OUT_VLD;   // [k][OUT_ULD]
  float* ssig = UsT + k * OUT_ULD;  // [k]
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  const int j0 = blockIdx.x * 256;
  for (int c = tid; c < k; c += 256) ssig[c] = float(sigma[c]);
  for (int e = tid; e < 256 * k; e += 256) {
    const int jj = e / k, c = e - jj * k;
    VsT[c * OUT_VLD + jj] = (j0 + jj < n) ? __ldg(V + int64_t(j0 + jj) * ldv + c) : 0.f;
  }
  const int j = j0 + 4 * tx;
  const bool vec = j + 3 < n && (ldx & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  for (int rt = 0; rt < OUT_RT; ++rt) {
    const int i0 = (blockIdx.y * OUT_RT + rt) * 32;
    if (i0 >= p) break;
    __syncthreads();  // VsT and ssig complete; UsT free for the next tile
    for (int e = tid; e < 32 * k; e += 256) {
      const int r = e / k, c = e - r * k;
      UsT[c * OUT_ULD + r] = (i0 + r < p) ? __ldg(U + int64_t(i0 + r) * ldu + c) * ssig[c] : 0.f;
    }
    __syncthreads();
    // packed pairs of rows: acc2[rp][q] = (acc[2 rp][q], acc[2 rp + 1][q])
    unsigned long long acc2[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc2[r][q] = 0ull;
    for (int c = 0; c < k; ++c) {
      const float4 u0 = *reinterpret_cast<const float4*>(UsT + c * OUT_ULD + 8 * ty);
      const float4 u1 = *reinterpret_cast<const float4*>(UsT + c * OUT_ULD + 8 * ty + 4);
      const float4 v = *reinterpret_cast<const float4*>(VsT + c * OUT_VLD + 4 * tx);
      unsigned long long up[4], vp[4];
      asm("mov.b64 %0, {%1, %2};" : "=l"(up[0]) : "f"(u0.x), "f"(u0.y));
      asm("mov.b64 %0, {%1, %2};" : "=l"(up[1]) : "f"(u0.z), "f"(u0.w));
      asm("mov.b64 %0, {%1, %2};" : "=l"(up[2]) : "f"(u1.x), "f"(u1.y));
      asm("mov.b64 %0, {%1, %2};" : "=l"(up[3]) : "f"(u1.z), "f"(u1.w));
      asm("mov.b64 %0, {%1, %1};" : "=l"(vp[0]) : "f"(v.x));
      asm("mov.b64 %0, {%1, %1};" : "=l"(vp[1]) : "f"(v.y));
      asm("mov.b64 %0, {%1, %1};" : "=l"(vp[2]) : "f"(v.z));
      asm("mov.b64 %0, {%1, %1};" : "=l"(vp[3]) : "f"(v.w));
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc2[r][q]) : "l"(up[r]), "l"(vp[q]));
    }
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[2 * r][q]), "=f"(acc[2 * r + 1][q]) : "l"(acc2[r][q]));
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + 8 * ty + r;
      if (i >= p) break;
      float* x = X + int64_t(i) * ldx + j;
      if (vec) {
        __stcs(reinterpret_cast<float4*>(x), make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j + q < n) __stcs(x + q, acc[r][q]);
      }
    }
  }
}

static size_t output_smem(int k) { return size_t(k) * (OUT_VLD + OUT_ULD + 1) * sizeof(float); }

// launch of output_kernel for a p x n X
static cpca_status launch_output(const float* U, int ldu, const float* V, int ldv, const double* sigma, int k,
                                 int p, int n, float* X, int64_t ldx, cudaStream_t st) {
  const size_t smem = output_smem(k);
  if (smem > 48 * 1024) {
    static PerDeviceOnce attr;
    CPCA_CUDA(once_per_device(attr, [&] {
      return cudaFuncSetAttribute(output_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(output_smem(KMAX_LIMIT)));
    }));
  }
  const dim3 og(ceil_div(n, 256), ceil_div(p, 32 * OUT_RT));
  output_kernel<<<og, 256, smem, st>>>(U, ldu, V, ldv, sigma, k, p, n, X, ldx);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

}  // namespace

struct DecodeWs {
  float *W, *Q, *Q2, *Ut, *Vt, *tn;
  double *G, *Rchol, *E, *lam, *s, *sinv, *rdiag;
  int* dead;
  int* k;
  int32_t *pos0, *pos1, *abar0, *abar1;
  float *minv0, *minv1;
  float* vec[2][6];
  double *acc, *acc_init;
  unsigned int* bar;
  int* err;
  int* out_iters;
  double* out_res;
  int* status;
  unsigned int* changed;
  int32_t *reach0, *reach1;
  int64_t *rp0, *rp1;
  int32_t *rcol0, *rcol1;
  float *rval0, *rval1;
  float *Ubuf, *Vbuf;
  double* sigbuf;
  double *npart_u, *npart_v, *invu, *invv;
  size_t bytes;
};

static int decode_block(int rr, int rc, int kmax) { return std::min(std::min(rr, rc), kmax + 8); }

static DecodeWs decode_layout(void* ws, int p, int n, int rr, int rc, int kmax, int64_t nnz_r,
                              int64_t nnz_c) {
  Carve c(ws);
  DecodeWs w{};
  const int b = decode_block(rr, rc, kmax);
  w.W = c.take<float>(size_t(std::max(rr, rc)) * b);
  w.Q = c.take<float>(size_t(std::max(rr, rc)) * b);
  w.Q2 = c.take<float>(size_t(std::max(rr, rc)) * b);
  w.Ut = c.take<float>(size_t(rr) * b);
  w.Vt = c.take<float>(size_t(rc) * b);
  w.G = c.take<double>(size_t(b) * b);
  w.tn = c.take<float>(skinny_scratch_floats(rr, rc, std::max(b, kmax)));
  w.Rchol = c.take<double>(size_t(b) * b);
  w.rdiag = c.take<double>(b);
  w.dead = c.take<int>(b);
  w.E = c.take<double>(size_t(b) * b);
  w.lam = c.take<double>(b);
  w.s = c.take<double>(b);
  w.sinv = c.take<double>(b);
  w.k = c.take<int>(1);
  w.pos0 = c.take<int32_t>(p);
  w.pos1 = c.take<int32_t>(n);
  const int m0 = p - rr, m1 = n - rc;
  w.abar0 = c.take<int32_t>(std::max(m0, 1));
  w.abar1 = c.take<int32_t>(std::max(m1, 1));
  w.minv0 = c.take<float>(std::max(m0, 1));
  w.minv1 = c.take<float>(std::max(m1, 1));
  for (int v = 0; v < 6; ++v) {
    w.vec[0][v] = c.take<float>(size_t(std::max(m0, 1)) * kmax);
    w.vec[1][v] = c.take<float>(size_t(std::max(m1, 1)) * kmax);
  }
  w.acc = c.take<double>(2 * 3 * 2 * KMAX_LIMIT);
  w.acc_init = c.take<double>(3 * 2 * KMAX_LIMIT);
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.out_iters = c.take<int>(2 * KMAX_LIMIT);
  w.out_res = c.take<double>(2 * KMAX_LIMIT);
  w.status = c.take<int>(1);
  w.changed = c.take<unsigned int>(3);
  w.rp0 = c.take<int64_t>(size_t(std::max(m0, 1)) + 1);
  w.rp1 = c.take<int64_t>(size_t(std::max(m1, 1)) + 1);
  w.rcol0 = c.take<int32_t>(std::max<int64_t>(nnz_r, 1));
  w.rcol1 = c.take<int32_t>(std::max<int64_t>(nnz_c, 1));
  w.rval0 = c.take<float>(std::max<int64_t>(nnz_r, 1));
  w.rval1 = c.take<float>(std::max<int64_t>(nnz_c, 1));
  w.reach0 = c.take<int32_t>(std::max(m0, 1));
  w.reach1 = c.take<int32_t>(std::max(m1, 1));
  w.Ubuf = c.take<float>(size_t(p) * kmax);
  w.Vbuf = c.take<float>(size_t(n) * kmax);
  w.sigbuf = c.take<double>(kmax);
  w.npart_u = c.take<double>(size_t(NORM_BLOCKS) * KMAX_LIMIT);
  w.npart_v = c.take<double>(size_t(NORM_BLOCKS) * KMAX_LIMIT);
  w.invu = c.take<double>(KMAX_LIMIT);
  w.invv = c.take<double>(KMAX_LIMIT);
  w.bytes = c.bytes();
  return w;
}

// Orthonormalise Q (m x b) in place by `passes` rank-revealing Cholesky-QR
// passes (two give orthogonality to working precision; one suffices inside
// the subspace iteration, where only the span matters).
static cpca_status orthonormalize(float* Q, float* Q2, int m, int b, int passes, const DecodeWs& w,
                                  cudaStream_t st) {
  for (int pass = 0; pass < passes; ++pass) {
    float* in = (pass & 1) ? Q2 : Q;
    float* out = (pass & 1) ? Q : Q2;
    CPCA_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * b * b, st));
    CPCA_PROF("svd_gram", st);
    gram_kernel<<<ceil_div(m, GRAM_ROWS), 256, 0, st>>>(in, m, b, w.G);
    CPCA_LAUNCHED();
    CPCA_PROF("svd_chol", st);
    chol_kernel<<<1, 256, 0, st>>>(w.G, b, w.Rchol, w.rdiag, w.dead);
    CPCA_LAUNCHED();
    trsm_rows_kernel<<<std::min<unsigned>(ceil_div(int64_t(m) * 32, 256), num_sms() * 8), 256, 0, st>>>(
        in, m, b, w.Rchol, w.rdiag, w.dead, out);
    CPCA_LAUNCHED();
  }
  if (passes & 1)
    CPCA_CUDA(cudaMemcpyAsync(Q, Q2, sizeof(float) * size_t(m) * b, cudaMemcpyDeviceToDevice, st));
  return CPCA_OK;
}

// Partial SVD of X~ (rr x rc) by block subspace iteration on the shorter
// side: S (short x b) <- orth((X~^T X~) S) or orth((X~ X~^T) S). Then
// T = X~ S (or X~^T S), Rayleigh-Ritz on T^T T = E diag(s~^2) E^T, and
// U~ = T E / s~, V~ = S E (or the mirror). Writes w.Ut (rr x b),
// w.Vt (rc x b), w.s, w.sinv, w.k.
static cpca_status partial_svd(const float* Xt, int rr, int rc, int64_t ldxt, int b, int iters,
                               uint64_t seed, double ratio, int k_override, const DecodeWs& w,
                               cudaStream_t st) {
  const bool vspace = rc <= rr;  // iterate on the columns' side
  const int ms = vspace ? rc : rr, ml = vspace ? rr : rc;
  float* Sb = w.W;   // short side, ms x b
  float* Sb2 = w.Q2; // scratch of at least ms x b
  float* T = w.Q;    // long side, ml x b
  auto to_long = [&](const float* in, float* out) -> cpca_status {
    CPCA_PROF("svd_gemm", st);
    if (vspace) {
      CPCA_TRY(nn_tall(Xt, ldxt, rr, rc, in, b, out, w.tn, st));
    } else {
      CPCA_TRY(tn_tall(Xt, ldxt, rr, rc, in, b, out, w.tn, st));
    }
    return CPCA_OK;
  };
  auto to_short = [&](const float* in, float* out) -> cpca_status {
    CPCA_PROF("svd_gemm", st);
    if (vspace) {
      CPCA_TRY(tn_tall(Xt, ldxt, rr, rc, in, b, out, w.tn, st));
    } else {
      CPCA_TRY(nn_tall(Xt, ldxt, rr, rc, in, b, out, w.tn, st));
    }
    return CPCA_OK;
  };
  const unsigned gs = std::min<unsigned>(ceil_div(int64_t(ms) * b, 256), num_sms() * 4);
  omega_kernel<<<gs, 256, 0, st>>>(Sb, ms, b, seed);
  CPCA_LAUNCHED();
  CPCA_TRY(orthonormalize(Sb, Sb2, ms, b, 1, w, st));
  for (int it = 0; it < iters; ++it) {
    CPCA_TRY(to_long(Sb, T));
    CPCA_TRY(to_short(T, Sb));
    CPCA_TRY(orthonormalize(Sb, Sb2, ms, b, it + 1 == iters ? 2 : 1, w, st));
  }
  CPCA_TRY(to_long(Sb, T));
  CPCA_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * b * b, st));
  CPCA_PROF("svd_gram", st);
  gram_kernel<<<ceil_div(ml, GRAM_ROWS), 256, 0, st>>>(T, ml, b, w.G);
  CPCA_LAUNCHED();
  CPCA_PROF("svd_jacobi", st);
  jacobi_eig_kernel<<<1, 256, 0, st>>>(w.G, b, w.E, w.lam);
  CPCA_LAUNCHED();
  rank_kernel<<<1, 32, 0, st>>>(w.lam, b, ratio, k_override, w.s, w.sinv, w.k);
  CPCA_LAUNCHED();
  const unsigned gl = std::min<unsigned>(ceil_div(int64_t(ml) * b, 256), num_sms() * 4);
  float* Ushort = vspace ? w.Vt : w.Ut;
  float* Ulong = vspace ? w.Ut : w.Vt;
  apply_small_kernel<<<gs, 256, 0, st>>>(Sb, ms, b, w.E, b, Ushort, b, nullptr);
  CPCA_LAUNCHED();
  apply_small_kernel<<<gl, 256, 0, st>>>(T, ml, b, w.E, b, Ulong, b, w.sinv);
  CPCA_LAUNCHED();
  (void)ml;
  return CPCA_OK;
}


// Sides 0 (U on Lr) and 1 (V on Lc) of the upsampling solves: index maps,
// the reduced L_aa CSR, and the PCG arguments over the workspace vectors.
// index_maps = false: the maps and the reduced CSR are already in the
// workspace (a forward call with the same inputs built them).
static cpca_status cg_setup(CgArgs& a, const cpca_csr* Lr, const cpca_csr* Lc, const int32_t* omega_r,
                            const int32_t* omega_c, int p, int n, int rr, int rc, int k, int b,
                            const cpca_decode_params* prm, const DecodeWs& w, cudaStream_t st,
                            bool index_maps = true, int sides = 3) {
  const CsrView lr{Lr->n, Lr->rowptr, Lr->col, Lr->val};
  const CsrView lc{Lc->n, Lc->rowptr, Lc->col, Lc->val};
  const int m[2] = {p - rr, n - rc};
  for (int sd = 0; sd < 2; ++sd) {
    CgSide& S = a.s[sd];
    S.N = sd ? n : p;
    S.rho = sd ? rc : rr;
    S.m = m[sd];
    S.L = sd ? lc : lr;
    S.omega = sd ? omega_c : omega_r;
    S.pos = sd ? w.pos1 : w.pos0;
    S.abar = sd ? w.abar1 : w.abar0;
    S.reach = sd ? w.reach1 : w.reach0;
    S.rp = sd ? w.rp1 : w.rp0;
    S.rcol = sd ? w.rcol1 : w.rcol0;
    S.rval = sd ? w.rval1 : w.rval0;
    S.minv = sd ? w.minv1 : w.minv0;
    S.R = sd ? w.Vt : w.Ut;
    S.ldr = b;
    S.rhs = nullptr;
    S.x = w.vec[sd][0];
    S.r = w.vec[sd][1];
    S.z = w.vec[sd][2];
    S.p0 = w.vec[sd][3];
    S.p1 = w.vec[sd][4];
    S.q = w.vec[sd][5];
    a.maxit[sd] = prm->cg_max_iter > 0 ? prm->cg_max_iter : 10 * std::max(m[sd], 1);
    if (!((sides >> sd) & 1)) {  // side left out: no nodes, no unknowns
      S.N = 0;
      S.rho = 0;
      S.m = 0;
    }
  }
  a.k = k;
  a.tol = prm->cg_tol;
  a.bar = grid_bar(w.bar, w.err);
  a.acc = w.acc;
  a.acc_init = w.acc_init;
  a.out_iters = w.out_iters;
  a.out_res = w.out_res;
  a.status = w.status;
  a.changed = w.changed;
  if (!index_maps) return CPCA_OK;
  dim3 sg(std::min<unsigned>(ceil_div(std::max(p, n), 256), num_sms() * 4), 2);
  cg_setup_kernel<<<sg, 256, 0, st>>>(a.s[0], a.s[1]);
  CPCA_LAUNCHED();
  laa_count_kernel<<<sg, 256, 0, st>>>(a.s[0], a.s[1]);
  CPCA_LAUNCHED();
  laa_scan_kernel<<<2, 1024, 0, st>>>(a.s[0], a.s[1]);
  CPCA_LAUNCHED();
  laa_fill_kernel<<<sg, 256, 0, st>>>(a.s[0], a.s[1]);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

// One cooperative PCG launch over both sides; synchronises and returns the
// per-column iteration counts, residuals and the status bits.
static cpca_status cg_solve(CgArgs& a, const DecodeWs& w, cudaStream_t st, int* cg_iters,
                            double* cg_res, int* breakdown) {
  CPCA_CUDA(cudaMemsetAsync(w.acc, 0, sizeof(double) * 2 * 3 * 2 * KMAX_LIMIT, st));
  CPCA_CUDA(cudaMemsetAsync(w.acc_init, 0, sizeof(double) * 3 * 2 * KMAX_LIMIT, st));
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, (kBarrierCounters + 1) * sizeof(unsigned int), st));
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  CPCA_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
  CPCA_CUDA(cudaMemsetAsync(w.changed, 0, 3 * sizeof(unsigned int), st));
  int occ = 0;
  CPCA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cg_kernel, 256, 0));
  const int64_t items = int64_t(a.s[0].m + a.s[1].m) * a.k;
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(occ) * num_sms(),
                                                               std::max<int64_t>(1, ceil_div(items, 256)))));
  void* args[] = {&a};
  CPCA_PROF("cg_pcg", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel((void*)cg_kernel, dim3(grid), dim3(256), args, 0, st));
  CPCA_LAUNCHED();
  int err = 0;
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(breakdown, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(cg_iters, w.out_iters, sizeof(int) * 2 * KMAX_LIMIT, cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(cg_res, w.out_res, sizeof(double) * 2 * KMAX_LIMIT, cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("cpca_decode: PCG grid barrier timed out");
    return CPCA_ERR_TIMEOUT;
  }
  return CPCA_OK;
}
// Lemma 1 on one graph for k given boundary columns: the minimiser of
// tr(S^T L S) subject to S(omega, :) = R (rho x k, ld ldr), by the decoder's
// Jacobi PCG (only its second side). Writes S (N x ldo, first k columns).
size_t harmonic_ws_bytes(int N, int rho, int k, int64_t nnz) {
  return decode_layout(nullptr, 1, N, 1, rho, k, 0, nnz).bytes;
}

cpca_status harmonic_extend(const cpca_csr* L, const int32_t* omega, int N, int rho, const float* R, int ldr,
                            int k, double tol, int maxit, float* S, int ldo, int* iters_max, double* res_max,
                            void* ws, cudaStream_t st) {
  CPCA_CHECK_ARG(k >= 1 && k <= KMAX_LIMIT && ldo >= k && ldr >= k, "harmonic extension: k %d", k);
  const DecodeWs w = decode_layout(ws, 1, N, 1, rho, k, 0, L->nnz);
  cpca_decode_params prm{};
  prm.cg_tol = tol;
  prm.cg_max_iter = maxit;
  prm.kmax = k;
  CgArgs a{};
  CPCA_TRY(cg_setup(a, L, L, omega, omega, 1, N, 1, rho, k, ldr, &prm, w, st, true, 2));
  a.s[1].R = R;
  a.s[1].ldr = ldr;
  int cg_iters[2 * KMAX_LIMIT] = {0};
  double cg_res[2 * KMAX_LIMIT] = {0};
  int breakdown = 0;
  CPCA_TRY(cg_solve(a, w, st, cg_iters, cg_res, &breakdown));
  const unsigned g = std::min<unsigned>(ceil_div(int64_t(N) * ldo, 256), num_sms() * 8);
  assemble_side_kernel<<<g, 256, 0, st>>>(N, k, ldo, w.pos1, R, ldr, w.vec[1][0], S);
  CPCA_LAUNCHED();
  int it = 0;
  double rs = 0.0;
  for (int c = 0; c < k; ++c) {
    it = std::max(it, cg_iters[KMAX_LIMIT + c]);
    rs = std::max(rs, cg_res[KMAX_LIMIT + c]);
  }
  if (iters_max) *iters_max = it;
  if (res_max) *res_max = rs;
  if (breakdown & 2) {
    set_error("harmonic extension: a connected component holds no sampled node");
    return CPCA_ERR_SINGULAR;
  }
  if (rs > tol) {
    set_error("harmonic extension: PCG stopped at relative residual %g", rs);
    return CPCA_ERR_NOT_CONVERGED;
  }
  return CPCA_OK;
}

// ---------------------------------------------------------- Kron reduction --
// L~ = L(O, O) - L(O, Ob) L(Ob, Ob)^-1 L(Ob, O) (Sec. IV-A) column by column:
// column j of L~ is (L h_j)(O), h_j the harmonic extension of the unit vector
// e_j given on the sampled nodes (h_j = e_j on O, -L_aa^-1 L_ab e_j on Ob).
// Chunks of up to KMAX_LIMIT columns go through the decoder's PCG at once.

// Sampled nodes strictly ascending and in [0, N).
__global__ void kron_omega_check_kernel(const int32_t* __restrict__ omega, int rho, int N, int* __restrict__ bad) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rho; t += gridDim.x * blockDim.x) {
    const int v = omega[t];
    if (v < 0 || v >= N || (t > 0 && omega[t - 1] >= v)) atomicOr(bad, 1);
  }
}

// R (rho x ldr): columns j0 .. j0 + kcur - 1 of the rho x rho identity, the
// rest of each row zero.
__global__ void kron_identity_kernel(float* __restrict__ R, int rho, int ldr, int j0, int kcur) {
  const int64_t total = int64_t(rho) * ldr;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / ldr), c = int(t % ldr);
    R[t] = (c < kcur && i == j0 + c) ? 1.f : 0.f;
  }
}

// Lt(i, j0 + c) = sum over row omega[i] of L of L(omega[i], t) h_c(t), with
// h_c(t) = x(pos[t], c) on unsampled t and [t is sampled node j0 + c] on
// sampled t; FP64 sum in CSR order.
__global__ void kron_cols_kernel(CsrView L, const int32_t* __restrict__ omega, const int32_t* __restrict__ pos,
                                 const float* __restrict__ x, int rho, int kcur, int j0, float* __restrict__ Lt,
                                 int64_t ldlt) {
  const int64_t total = int64_t(rho) * kcur;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / kcur), c = int(t % kcur);
    const int node = omega[i];
    double v = 0.0;
    for (int64_t e = L.rowptr[node]; e < L.rowptr[node + 1]; ++e) {
      const int ps = pos[L.col[e]];
      const double h = ps >= 0 ? double(x[int64_t(ps) * kcur + c]) : ((-ps - 1) == j0 + c ? 1.0 : 0.0);
      v += double(L.val[e]) * h;
    }
    Lt[int64_t(i) * ldlt + j0 + c] = float(v);
  }
}

// Lt <- (Lt + Lt^T) / 2 in place: the thread of (i, j), i < j, owns the pair.
__global__ void kron_sym_kernel(float* __restrict__ Lt, int64_t ld, int rho) {
  const int64_t total = int64_t(rho) * rho;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / rho), j = int(t % rho);
    if (i < j) {
      float* a = Lt + int64_t(i) * ld + j;
      float* b = Lt + int64_t(j) * ld + i;
      const float m = 0.5f * (*a + *b);
      *a = m;
      *b = m;
    }
  }
}

// The dense rho x rho matrix as CSR with every entry stored.
__global__ void kron_csr_kernel(const float* __restrict__ Lt, int64_t ld, int rho, int64_t* __restrict__ rowptr,
                                int32_t* __restrict__ col, float* __restrict__ val) {
  const int64_t total = int64_t(rho) * rho;
  const int64_t g0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x, gs = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = g0; t < total; t += gs) {
    const int i = int(t / rho), j = int(t % rho);
    col[t] = j;
    val[t] = Lt[int64_t(i) * ld + j];
  }
  for (int64_t t = g0; t <= rho; t += gs) rowptr[t] = t * rho;
}

struct KronWs {
  DecodeWs d;
  float* R;
  int* bad;
  size_t bytes;
};

static KronWs kron_layout(void* ws, int N, int rho, int64_t nnz) {
  const int kc = std::min(rho, KMAX_LIMIT);
  KronWs k{};
  k.d = decode_layout(ws, 1, N, 1, rho, kc, 0, nnz);
  Carve c(ws ? static_cast<char*>(ws) + k.d.bytes : nullptr);
  k.R = c.take<float>(size_t(rho) * kc);
  k.bad = c.take<int>(1);
  k.bytes = k.d.bytes + c.bytes();
  return k;
}

}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_decode_workspace_size(int32_t p, int32_t n, int32_t rr, int32_t rc, int32_t kmax,
                                             int64_t nnz_r, int64_t nnz_c) {
  if (p <= 0 || n <= 0 || rr <= 0 || rc <= 0 || kmax <= 0 || kmax > KMAX_LIMIT || nnz_r < 0 || nnz_c < 0)
    return 0;
  return decode_layout(nullptr, p, n, rr, rc, kmax, nnz_r, nnz_c).bytes;
}

extern "C" cpca_status cpca_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                   const int32_t* omega_r, const int32_t* omega_c, int32_t p,
                                   int32_t n, const cpca_csr* Lr, const cpca_csr* Lc,
                                   const cpca_decode_params* prm, float* X, int64_t ldx, float* U,
                                   float* V, double* sigma, int32_t* k_out, cpca_decode_info* info,
                                   void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_decode");
  CPCA_CHECK_ARG(Xt && omega_r && omega_c && prm, "cpca_decode: null pointer");
  CPCA_CHECK_ARG(rr > 0 && rc > 0 && rr <= p && rc <= n, "cpca_decode: need 0 < rr <= p, 0 < rc <= n");
  CPCA_CHECK_ARG(ldxt >= rc, "cpca_decode: ldxt < rc");
  CPCA_CHECK_ARG(!X || ldx >= n, "cpca_decode: ldx < n");
  CPCA_CHECK_ARG(prm->kmax >= 1 && prm->kmax <= KMAX_LIMIT, "cpca_decode: kmax must be in [1, %d]", KMAX_LIMIT);
  CPCA_CHECK_ARG(prm->delta >= 0 && prm->delta < 1, "cpca_decode: delta must be in [0, 1)");
  CPCA_CHECK_ARG(prm->cg_tol > 0, "cpca_decode: cg_tol must be positive");
  CPCA_CHECK_ARG(prm->svd_iters >= 1, "cpca_decode: svd_iters < 1");
  CPCA_CHECK_ARG(prm->rank_ratio > 0 && prm->rank_ratio <= 1, "cpca_decode: rank_ratio in (0, 1]");
  CPCA_TRY(check_csr(Lr, p, "cpca_decode(Lr)"));
  CPCA_TRY(check_csr(Lc, n, "cpca_decode(Lc)"));
  const int kmax = prm->kmax;
  const DecodeWs w = decode_layout(ws, p, n, rr, rc, kmax, Lr->nnz, Lc->nnz);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_decode: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int b = decode_block(rr, rc, kmax);
  CPCA_TRY(partial_svd(Xt, rr, rc, ldxt, b, prm->svd_iters, prm->svd_seed, prm->rank_ratio,
                       prm->k_override, w, st));
  int k = 0;
  CPCA_CUDA(cudaMemcpyAsync(&k, w.k, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (k > kmax || k > b) {
    set_error("cpca_decode: rank %d exceeds kmax %d or block %d", k, kmax, b);
    return CPCA_ERR_INVALID_ARG;
  }
  float* Uo = U ? U : w.Ubuf;
  float* Vo = V ? V : w.Vbuf;
  double* so = sigma ? sigma : w.sigbuf;
  int cg_iters[2 * KMAX_LIMIT] = {0};
  double cg_res[2 * KMAX_LIMIT] = {0};
  int breakdown = 0;
  if (k > 0) {
    CgArgs a{};
    CPCA_TRY(cg_setup(a, Lr, Lc, omega_r, omega_c, p, n, rr, rc, k, b, prm, w, st));
    CPCA_TRY(cg_solve(a, w, st, cg_iters, cg_res, &breakdown));
  }
  // assemble, normalise, scale, output
  const unsigned gp = std::min<unsigned>(ceil_div(int64_t(p) * kmax, 256), num_sms() * 8);
  const unsigned gn = std::min<unsigned>(ceil_div(int64_t(n) * kmax, 256), num_sms() * 8);
  assemble_side_kernel<<<gp, 256, 0, st>>>(p, k, kmax, w.pos0, w.Ut, b, w.vec[0][0], Uo);
  CPCA_LAUNCHED();
  assemble_side_kernel<<<gn, 256, 0, st>>>(n, k, kmax, w.pos1, w.Vt, b, w.vec[1][0], Vo);
  CPCA_LAUNCHED();
  if (k == 0) {
    // no singular value: X = 0; pos maps were not built, so overwrite
    CPCA_CUDA(cudaMemsetAsync(Uo, 0, sizeof(float) * size_t(p) * kmax, st));
    CPCA_CUDA(cudaMemsetAsync(Vo, 0, sizeof(float) * size_t(n) * kmax, st));
  }
  colnorm_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(Uo, p, k, kmax, w.npart_u);
  CPCA_LAUNCHED();
  colnorm_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(Vo, n, k, kmax, w.npart_v);
  CPCA_LAUNCHED();
  const double scale = sqrt(double(n) * double(p) / (double(rr) * double(rc) * (1.0 - prm->delta)));
  norm_finish_kernel<<<1, 64, 0, st>>>(w.npart_u, w.npart_v, NORM_BLOCKS, k, w.s, scale, w.invu,
                                       w.invv, so, kmax);
  CPCA_LAUNCHED();
  scale_cols_kernel<<<gp, 256, 0, st>>>(Uo, int64_t(p) * kmax, kmax, w.invu);
  CPCA_LAUNCHED();
  scale_cols_kernel<<<gn, 256, 0, st>>>(Vo, int64_t(n) * kmax, kmax, w.invv);
  CPCA_LAUNCHED();
  if (X) {  // device memory, or page-locked host memory the GPU addresses (written by the kernel)
    CPCA_PROF("decode_output", st);
    CPCA_TRY(launch_output(Uo, kmax, Vo, kmax, so, k, p, n, X, ldx, st));  // k == 0: zeros
  }
  if (k_out) *k_out = k;
  int itmax[2] = {0, 0};
  double resmax[2] = {0, 0};
  bool capped = false;
  for (int sd = 0; sd < 2; ++sd)
    for (int c = 0; c < k; ++c) {
      itmax[sd] = std::max(itmax[sd], cg_iters[sd * KMAX_LIMIT + c]);
      resmax[sd] = std::max(resmax[sd], cg_res[sd * KMAX_LIMIT + c]);
      if (cg_res[sd * KMAX_LIMIT + c] > prm->cg_tol) capped = true;
    }
  if (info) {
    CPCA_CUDA(cudaMemcpyAsync(info->s_tilde, w.s, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));
    info->k = k;
    info->b = b;
    info->cg_iters_u = itmax[0];
    info->cg_iters_v = itmax[1];
    info->cg_res_u = resmax[0];
    info->cg_res_v = resmax[1];
  }
  if (breakdown) {
    set_error("cpca_decode: L_aa is not positive definite (a graph component has no sampled node)");
    return CPCA_ERR_SINGULAR;
  }
  if (capped) {
    set_error("cpca_decode: PCG reached cg_max_iter before cg_tol");
    return CPCA_ERR_NOT_CONVERGED;
  }
  return CPCA_OK;
}

// ===================================================================== //
// Reverse mode of the decoder (the paper has no derivatives; this is the  //
// derivative of the computed map with k fixed).                           //
//                                                                         //
// Forward: (U~, s, V~) = top-k SVD of X~; Uh = extension of U~ on Lr      //
// (Lemma 1: Uh(Omega) = U~, Uh(a) = -Lr_aa^-1 Lr_ab U~), U = Uh / |Uh|    //
// column-wise, sigma = c s; likewise V; X = U diag(sigma) V^T.            //
// Given dloss/dX at entries (i_e, j_e): Ub, Vb, sigmab by scattering;     //
// Uhb = (Ub - U diag(U^T Ub)) / |Uh|; Lambda = Lr_aa^-1 Uhb(a) (adjoint   //
// PCG, Lr_aa symmetric); U~b = Uhb(Omega) - Lr_{a,Omega}^T Lambda;        //
// dLr(i, j) = -sum_c Lambda(i, c) Uh(j, c) for unsampled rows i.          //
// SVD: with A = X~ (or X~^T so that A is m x n, m >= n), J_u = U^T Ub,    //
// J_v = V^T Vb, F_ij = 1 / (s_j^2 - s_i^2):                               //
//   Ab = U Cm V^T + E V^T + U F'^T,                                       //
//   Cm_ij = F_ij (J_u - J_u^T)_ij s_j + delta_ij sb_i + s_i F_ij (J_v - J_v^T)_ij, //
// and the parts outside the top-k subspaces through the resolvents of the //
// Gram G = A^T A restricted to the complement of V (SPD there, shift s_i^2 //
// above the discarded spectrum):                                          //
//   B = Ub - U J_u, y'_i = (s_i^2 - G)^-1 A^T b_i, y_i = (s_i^2 - G)^-1 d_i, //
//   d_i = vb_i - V (J_v)_i, E = B S^-1 + A (Y' S^-1 + Y), F' = Y' + Y S.   //
// The shifted systems are solved by dense CG, one block per right-hand    //
// side; the same identity (Woodbury) replaces the m x m resolvent.        //
// ===================================================================== //
namespace cpca {
namespace {

__global__ void heldout_kernel(int64_t nh, const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                               const float* __restrict__ g, const float* __restrict__ U,
                               const float* __restrict__ V, int ld, const double* __restrict__ sigma, int k,
                               float* __restrict__ Ub, float* __restrict__ Vb, double* __restrict__ sbar) {
  __shared__ double sb[KMAX_LIMIT];
  for (int c = threadIdx.x; c < KMAX_LIMIT; c += blockDim.x) sb[c] = 0.0;
  __syncthreads();
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nh;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int i = rows[e], j = cols[e];
    const double ge = g[e];
    for (int c = 0; c < k; ++c) {
      const double u = U[int64_t(i) * ld + c], v = V[int64_t(j) * ld + c], s = sigma[c];
      atomicAdd(Ub + int64_t(i) * ld + c, float(ge * s * v));
      atomicAdd(Vb + int64_t(j) * ld + c, float(ge * s * u));
      atomicAdd(sb + c, ge * u * v);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x)
    if (sb[c] != 0.0) atomicAdd(sbar + c, sb[c]);
}

// Column-wise FP64 dot products of A and B (N x k, ld), fixed order per block.
__global__ void coldot_partial_kernel(const float* __restrict__ A, const float* __restrict__ B, int N, int k,
                                      int ld, double* __restrict__ part) {
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(N, lo + per);
  const int c = threadIdx.x % KMAX_LIMIT, lane_row = threadIdx.x / KMAX_LIMIT;
  const int rows_par = blockDim.x / KMAX_LIMIT;
  double acc = 0.0;
  if (c < k && lane_row < rows_par)
    for (int i = lo + lane_row; i < hi; i += rows_par)
      acc += double(A[int64_t(i) * ld + c]) * double(B[int64_t(i) * ld + c]);
  __shared__ double tmp[256];
  tmp[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < KMAX_LIMIT) {
    double t = 0.0;
    for (int r = 0; r < rows_par; ++r) t += tmp[r * KMAX_LIMIT + threadIdx.x];
    part[int64_t(blockIdx.x) * KMAX_LIMIT + threadIdx.x] = t;
  }
}
__global__ void sum_parts_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  for (int c = threadIdx.x; c < KMAX_LIMIT; c += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nblk; ++i) a += part[int64_t(i) * KMAX_LIMIT + c];
    out[c] = a;
  }
}

// Ub <- (Ub - U diag(dots)) diag(inv): adjoint of the column normalisation.
__global__ void norm_bwd_kernel(float* __restrict__ Ub, const float* __restrict__ U, int64_t total, int ld,
                                int k, const double* __restrict__ dots, const double* __restrict__ inv) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t % ld);
    Ub[t] = c < k ? float((double(Ub[t]) - double(U[t]) * dots[c]) * inv[c]) : 0.f;
  }
}

__global__ void gather_rhs_kernel(int m, int k, const int32_t* __restrict__ abar, const float* __restrict__ X,
                                  int ld, float* __restrict__ rhs) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(m) * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / k), c = int(t % k);
    rhs[t] = X[int64_t(abar[r]) * ld + c];
  }
}

// R~b(s, c) = Uhb(omega_s, c) - sum_{j unsampled} L(omega_s, j) Lambda(pos_j, c).
__global__ void sampled_bar_kernel(int rho, const int32_t* __restrict__ omega, CsrView L,
                                   const int32_t* __restrict__ pos, const float* __restrict__ Uhb, int ld,
                                   const float* __restrict__ Lam, int k, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(rho) * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int s = int(t / k), c = int(t % k);
    const int node = omega[s];
    double v = Uhb[int64_t(node) * ld + c];
    for (int64_t e = L.rowptr[node]; e < L.rowptr[node + 1]; ++e) {
      const int ps = pos[L.col[e]];
      if (ps >= 0) v -= double(L.val[e]) * double(Lam[int64_t(ps) * k + c]);
    }
    out[t] = float(v);
  }
}

// dL(e) for e = (i, j): -sum_c Lambda(pos_i, c) Uh(j, c) if i is unsampled, else 0.
__global__ void dl_decode_kernel(CsrView L, const int32_t* __restrict__ pos, const float* __restrict__ Lam,
                                 int k, const float* __restrict__ Uh, int ld, double* __restrict__ dL) {
  for (int i = blockIdx.x; i < L.n; i += gridDim.x) {
    const int t = pos[i];
    for (int64_t e = L.rowptr[i] + threadIdx.x; e < L.rowptr[i + 1]; e += blockDim.x) {
      double v = 0.0;
      if (t >= 0) {
        const int j = L.col[e];
        for (int c = 0; c < k; ++c) v -= double(Lam[int64_t(t) * k + c]) * double(Uh[int64_t(j) * ld + c]);
      }
      dL[e] = v;
    }
  }
}

// out (k x k, FP64, zeroed) += P^T Q over m rows (P, Q with their own ld).
__global__ void cross_gram_kernel(const float* __restrict__ P, int ldp, const float* __restrict__ Q, int ldq,
                                  int m, int k, double* __restrict__ out) {
  const int r0 = blockIdx.x * 64, r1 = min(m, r0 + 64);
  for (int pr = threadIdx.x; pr < k * k; pr += blockDim.x) {
    const int i = pr / k, j = pr % k;
    double s = 0.0;
    for (int t = r0; t < r1; ++t) s += double(P[int64_t(t) * ldp + i]) * double(Q[int64_t(t) * ldq + j]);
    if (s != 0.0) atomicAdd(out + pr, s);
  }
}

// Cm (k x k) of the in-subspace part; sb = scale * sigmab.
__global__ void svd_mid_kernel(int k, const double* __restrict__ s, const double* __restrict__ sigb, double scale,
                               const double* __restrict__ Ju, const double* __restrict__ Jv,
                               double* __restrict__ Cm) {
  for (int pr = threadIdx.x; pr < k * k; pr += blockDim.x) {
    const int i = pr / k, j = pr % k;
    double v = 0.0;
    if (i == j) {
      v = scale * sigb[i];
    } else {
      const double den = s[j] * s[j] - s[i] * s[i];
      if (den != 0.0) {
        const double F = 1.0 / den;
        v = F * (Ju[i * k + j] - Ju[j * k + i]) * s[j] + s[i] * F * (Jv[i * k + j] - Jv[j * k + i]);
      }
    }
    Cm[pr] = v;
  }
}

// out (m x k) = Pb - Ubase J (J k x k FP64); Ubase with ld ldu, Pb and out ld k.
__global__ void proj_sub_kernel(int m, int k, const float* __restrict__ Pb, const float* __restrict__ Ub, int ldu,
                                const double* __restrict__ J, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(m) * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / k), i = int(t % k);
    double v = Pb[t];
    for (int j = 0; j < k; ++j) v -= double(Ub[int64_t(r) * ldu + j]) * J[j * k + i];
    out[t] = float(v);
  }
}

// G (n x n, FP32) = A^T A with A = X~ (rows t, columns a) when vspace, else
// A = X~^T. 32 x 32 output tile per block, FP32 products per 32-chunk of
// the summed dimension, FP64 across chunks.
__global__ void __launch_bounds__(256)
gram_full_kernel(const float* __restrict__ X, int64_t ldx, int rr, int rc, int vspace, float* __restrict__ G) {
  __shared__ float As[32][33], Bs[32][33];
  const int n = vspace ? rc : rr, m = vspace ? rr : rc;
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4 outputs each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = 0; t0 < m; t0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int tt = e >> 5, cc = e & 31;
      float va = 0.f, vb = 0.f;
      if (vspace) {
        if (t0 + tt < m && a0 + cc < n) va = X[int64_t(t0 + tt) * ldx + a0 + cc];
        if (t0 + tt < m && b0 + cc < n) vb = X[int64_t(t0 + tt) * ldx + b0 + cc];
        As[tt][cc] = va;
        Bs[tt][cc] = vb;
      } else {
        // element (t, a) of A = X~(a, t): read along t
        if (t0 + cc < m && a0 + tt < n) va = X[int64_t(a0 + tt) * ldx + t0 + cc];
        if (t0 + cc < m && b0 + tt < n) vb = X[int64_t(b0 + tt) * ldx + t0 + cc];
        As[cc][tt] = va;
        Bs[cc][tt] = vb;
      }
    }
    __syncthreads();
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int tt = 0; tt < 32; ++tt) {
      const float bv = Bs[tt][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) part[q] = fmaf(As[tt][ty * 4 + q], bv, part[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += part[q];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ty * 4 + q, b = b0 + tx;
    if (a < n && b < n) G[int64_t(a) * n + b] = float(acc[q]);
  }
}

// vec (n, global) <- vec - V (V^T vec), V n x k with ld ldv.
__device__ __forceinline__ void project_out(float* vec, const float* __restrict__ V, int ldv, int k, int n,
                                            double* red) {
  for (int c = 0; c < k; ++c) {
    __syncthreads();
    double d = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) d += double(V[int64_t(a) * ldv + c]) * vec[a];
    d = block_sum(d, red);
    for (int a = threadIdx.x; a < n; a += blockDim.x) vec[a] = float(double(vec[a]) - d * V[int64_t(a) * ldv + c]);
  }
  __syncthreads();
}

// (s_i^2 I - G) y = rhs on the complement of V (n x k, ld ldv), one block
// per right-hand side; right-hand side r < k uses rhs0 column r, else rhs1
// column r - k (both n x k); shift s_{r mod k}^2. CG on the projected
// operator P (s^2 I - G) P, P = I - V V^T (SPD on the complement; the
// top-k directions of the computed basis are only approximately invariant,
// so every product is projected), FP64 scalars.
__global__ void __launch_bounds__(256)
shift_cg_kernel(const float* __restrict__ G, int n, int k, const float* __restrict__ rhs0,
                const float* __restrict__ rhs1, const double* __restrict__ s, const float* __restrict__ V,
                int ldv, double tol, int maxit, float* __restrict__ work, float* __restrict__ out0,
                float* __restrict__ out1, int* __restrict__ flag) {
  extern __shared__ float ps[];
  __shared__ double red[8];
  const int r = blockIdx.x;
  const float* rhs = r < k ? rhs0 : rhs1;
  float* out = r < k ? out0 : out1;
  const int col = r < k ? r : r - k;
  const float shift = float(s[col] * s[col]);
  float* x = work + int64_t(r) * 3 * n;
  float* res = x + n;
  float* q = res + n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    x[a] = 0.f;
    res[a] = rhs[int64_t(a) * k + col];
  }
  project_out(res, V, ldv, k, n, red);
  double bb = 0.0;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    ps[a] = res[a];
    bb += double(res[a]) * res[a];
  }
  bb = block_sum(bb, red);
  double rr = bb;
  const double stop = tol * tol * bb;
  int it = 0;
  while (rr > stop && it < maxit) {
    __syncthreads();
    for (int a = warp; a < n; a += 8) {
      float sum = 0.f;
      for (int b = lane; b < n; b += 32) sum = fmaf(G[int64_t(a) * n + b], ps[b], sum);
      sum = warp_sumf(sum);
      if (lane == 0) q[a] = shift * ps[a] - sum;
    }
    project_out(q, V, ldv, k, n, red);
    double pq = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) pq += double(ps[a]) * q[a];
    pq = block_sum(pq, red);
    if (!(pq > 0.0)) {
      if (threadIdx.x == 0) atomicOr(flag, 1);
      break;
    }
    const double alpha = rr / pq;
    double rn = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
      x[a] = float(double(x[a]) + alpha * ps[a]);
      const float rv = float(double(res[a]) - alpha * q[a]);
      res[a] = rv;
      rn += double(rv) * rv;
    }
    rn = block_sum(rn, red);
    const double beta = rn / rr;
    rr = rn;
    for (int a = threadIdx.x; a < n; a += blockDim.x) ps[a] = float(res[a] + beta * ps[a]);
    ++it;
  }
  if (rr > stop && threadIdx.x == 0) atomicOr(flag, 2);
  project_out(x, V, ldv, k, n, red);
  for (int a = threadIdx.x; a < n; a += blockDim.x) out[int64_t(a) * k + col] = x[a];
}

// T = Y' S^-1 + Y and F' = Y' + Y S (n x k).
__global__ void tcomb_kernel(int n, int k, const float* __restrict__ Yp, const float* __restrict__ Yv,
                             const double* __restrict__ s, float* __restrict__ T, float* __restrict__ F) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(n) * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t % k);
    T[t] = float(double(Yp[t]) / s[i] + Yv[t]);
    F[t] = float(Yp[t] + double(Yv[t]) * s[i]);
  }
}

// P = U Cm + B S^-1 + AT (m x k).
__global__ void pcomb_kernel(int m, int k, const float* __restrict__ U, int ldu, const double* __restrict__ Cm,
                             const float* __restrict__ B, const float* __restrict__ AT,
                             const double* __restrict__ s, float* __restrict__ P) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(m) * k;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / k), i = int(t % k);
    double v = double(B[t]) / s[i] + AT[t];
    for (int j = 0; j < k; ++j) v += double(U[int64_t(r) * ldu + j]) * Cm[j * k + i];
    P[t] = float(v);
  }
}

// Ab (m x n) = P V^T + U F'^T, written as X~b (transposed when A = X~^T).
__global__ void __launch_bounds__(256)
lowrank_out_kernel(int m, int n, int k, const float* __restrict__ P, const float* __restrict__ V, int ldv,
                   const float* __restrict__ U, int ldu, const float* __restrict__ F, float* __restrict__ out,
                   int64_t ldo, int transposed) {
  __shared__ float Ps[32][2 * KMAX_LIMIT + 1];
  __shared__ float Qs[32][2 * KMAX_LIMIT + 1];
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    const bool ia = a0 + r < m, ib = b0 + r < n;
    Ps[r][c] = ia ? P[int64_t(a0 + r) * k + c] : 0.f;
    Ps[r][k + c] = ia ? U[int64_t(a0 + r) * ldu + c] : 0.f;
    Qs[r][c] = ib ? V[int64_t(b0 + r) * ldv + c] : 0.f;
    Qs[r][k + c] = ib ? F[int64_t(b0 + r) * k + c] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    const int ra = ty * 4 + q;
    // transposed output: lanes run along a (rows of A) for coalesced stores
    const int ia = transposed ? tx : ra, ib = transposed ? ra : tx;
    const int a = a0 + ia, b = b0 + ib;
    if (a >= m || b >= n) continue;
    float v = 0.f;
    for (int c = 0; c < 2 * k; ++c) v = fmaf(Ps[ia][c], Qs[ib][c], v);
    if (transposed) out[int64_t(b) * ldo + a] = v;
    else out[int64_t(a) * ldo + b] = v;
  }
}

// X(h_row[e], h_col[e]) = sum_c U(i, c) sigma_c V(j, c), FP64 sum.
__global__ void entries_kernel(int64_t nh, const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                               const float* __restrict__ U, int ldu, const float* __restrict__ V, int ldv,
                               const double* __restrict__ sigma, int k, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nh;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int i = rows[e], j = cols[e];
    double v = 0.0;
    for (int c = 0; c < k; ++c) v += double(U[int64_t(i) * ldu + c]) * sigma[c] * double(V[int64_t(j) * ldv + c]);
    out[e] = float(v);
  }
}

struct DecBwdWs {
  float *Uh, *Vh, *Ub, *Vb;
  double *sbar, *part, *dots_u, *dots_v;
  float *rhs0, *rhs1;
  float *Utb, *Vtb;
  double *Ju, *Jv, *Cm;
  float *B, *Cc, *D, *Yp, *Yv, *T, *F, *AT, *P, *G, *work;
  double *dL0, *dL1, *deg, *dD;
  int* flag;
  size_t bytes;
};

DecBwdWs decbwd_layout(void* base, int p, int n, int rr, int rc, int kmax, int64_t nnz_r, int64_t nnz_c) {
  Carve c(base);
  DecBwdWs w{};
  const int ma = std::max(rr, rc), na = std::min(rr, rc);
  w.Uh = c.take<float>(size_t(p) * kmax);
  w.Vh = c.take<float>(size_t(n) * kmax);
  w.Ub = c.take<float>(size_t(p) * kmax);
  w.Vb = c.take<float>(size_t(n) * kmax);
  w.sbar = c.take<double>(KMAX_LIMIT);
  w.part = c.take<double>(size_t(NORM_BLOCKS) * KMAX_LIMIT);
  w.dots_u = c.take<double>(KMAX_LIMIT);
  w.dots_v = c.take<double>(KMAX_LIMIT);
  w.rhs0 = c.take<float>(size_t(std::max(p - rr, 1)) * kmax);
  w.rhs1 = c.take<float>(size_t(std::max(n - rc, 1)) * kmax);
  w.Utb = c.take<float>(size_t(rr) * kmax);
  w.Vtb = c.take<float>(size_t(rc) * kmax);
  w.Ju = c.take<double>(size_t(kmax) * kmax);
  w.Jv = c.take<double>(size_t(kmax) * kmax);
  w.Cm = c.take<double>(size_t(kmax) * kmax);
  w.B = c.take<float>(size_t(ma) * kmax);
  w.Cc = c.take<float>(size_t(na) * kmax);
  w.D = c.take<float>(size_t(na) * kmax);
  w.Yp = c.take<float>(size_t(na) * kmax);
  w.Yv = c.take<float>(size_t(na) * kmax);
  w.T = c.take<float>(size_t(na) * kmax);
  w.F = c.take<float>(size_t(na) * kmax);
  w.AT = c.take<float>(size_t(ma) * kmax);
  w.P = c.take<float>(size_t(ma) * kmax);
  w.G = c.take<float>(size_t(na) * na);
  w.work = c.take<float>(size_t(2 * kmax) * 3 * na);
  w.dL0 = c.take<double>(std::max<int64_t>(nnz_r, 1));
  w.dL1 = c.take<double>(std::max<int64_t>(nnz_c, 1));
  w.deg = c.take<double>(std::max(p, n));
  w.dD = c.take<double>(std::max(p, n));
  w.flag = c.take<int>(1);
  w.bytes = c.bytes();
  return w;
}

constexpr int kShiftCgMaxN = 16384;  // dense resolvent solves keep p in shared memory

}  // namespace
}  // namespace cpca

extern "C" size_t cpca_decode_backward_workspace_size(int32_t p, int32_t n, int32_t rr, int32_t rc,
                                                      int32_t kmax, int64_t nnz_r, int64_t nnz_c) {
  const size_t a = cpca_decode_workspace_size(p, n, rr, rc, kmax, nnz_r, nnz_c);
  if (a == 0) return 0;
  const size_t fwd = (a + 255) & ~size_t(255);
  return fwd + decbwd_layout(nullptr, p, n, rr, rc, kmax, nnz_r, nnz_c).bytes;
}

extern "C" cpca_status cpca_decode_backward(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                            const int32_t* omega_r, const int32_t* omega_c, int32_t p,
                                            int32_t n, const cpca_csr* Lr, const cpca_csr* Lc,
                                            const cpca_decode_params* prm, int32_t k, int32_t resume,
                                            int64_t nh,
                                            const int32_t* h_row, const int32_t* h_col,
                                            const float* h_grad, float* dXt, int64_t lddxt, double* dLr,
                                            double* dLc, const float* wr, const float* wc,
                                            int32_t lap_type, float* dwr, float* dwc, void* ws,
                                            size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_decode_backward");
  CPCA_CHECK_ARG(Xt && omega_r && omega_c && prm && dXt, "cpca_decode_backward: null pointer");
  CPCA_CHECK_ARG(nh >= 0 && (nh == 0 || (h_row && h_col && h_grad)), "cpca_decode_backward: bad entries");
  CPCA_CHECK_ARG(rr > 0 && rc > 0 && rr <= p && rc <= n, "cpca_decode_backward: need 0 < rr <= p, 0 < rc <= n");
  CPCA_CHECK_ARG(ldxt >= rc && lddxt >= rc, "cpca_decode_backward: leading dimension < rc");
  CPCA_CHECK_ARG(prm->kmax >= 1 && prm->kmax <= KMAX_LIMIT, "cpca_decode_backward: kmax must be in [1, %d]",
                 KMAX_LIMIT);
  CPCA_CHECK_ARG(k >= 1 && k <= prm->kmax, "cpca_decode_backward: need 1 <= k <= kmax");
  CPCA_CHECK_ARG(prm->delta >= 0 && prm->delta < 1, "cpca_decode_backward: delta must be in [0, 1)");
  CPCA_CHECK_ARG(prm->cg_tol > 0 && prm->svd_iters >= 1, "cpca_decode_backward: bad cg_tol / svd_iters");
  CPCA_CHECK_ARG(lap_type == CPCA_LAP_NORMALIZED || lap_type == CPCA_LAP_COMBINATORIAL,
                 "cpca_decode_backward: unknown lap_type");
  CPCA_CHECK_ARG(!dwr || wr, "cpca_decode_backward: dwr needs the weights wr");
  CPCA_CHECK_ARG(!dwc || wc, "cpca_decode_backward: dwc needs the weights wc");
  CPCA_CHECK_ARG(std::min(rr, rc) <= kShiftCgMaxN, "cpca_decode_backward: min(rr, rc) > %d", kShiftCgMaxN);
  CPCA_TRY(check_csr(Lr, p, "cpca_decode_backward(Lr)"));
  CPCA_TRY(check_csr(Lc, n, "cpca_decode_backward(Lc)"));
  const int kmax = prm->kmax;
  const DecodeWs w = decode_layout(ws, p, n, rr, rc, kmax, Lr->nnz, Lc->nnz);
  const size_t fwd = (w.bytes + 255) & ~size_t(255);
  const DecBwdWs v = decbwd_layout(ws ? static_cast<char*>(ws) + fwd : nullptr, p, n, rr, rc, kmax, Lr->nnz,
                                   Lc->nnz);
  if (!ws || ws_bytes < fwd + v.bytes) {
    set_error("cpca_decode_backward: workspace %zu bytes < required %zu", ws_bytes, fwd + v.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int b = decode_block(rr, rc, kmax);
  CPCA_CHECK_ARG(k <= b, "cpca_decode_backward: k > subspace block %d", b);
  // ---- forward factors, k fixed (resume: the forward call left them in ws)
  CgArgs a{};
  int cg_iters[2 * KMAX_LIMIT] = {0};
  double cg_res[2 * KMAX_LIMIT] = {0};
  int breakdown = 0;
  if (resume) {
    int kf = 0;
    CPCA_CUDA(cudaMemcpyAsync(&kf, w.k, sizeof(int), cudaMemcpyDeviceToHost, st));
    CPCA_CUDA(cudaStreamSynchronize(st));
    CPCA_CHECK_ARG(kf == k, "cpca_decode_backward: resume with k = %d, but the forward found k = %d", k, kf);
    CPCA_TRY(cg_setup(a, Lr, Lc, omega_r, omega_c, p, n, rr, rc, k, b, prm, w, st, false));
  } else {
    CPCA_TRY(partial_svd(Xt, rr, rc, ldxt, b, prm->svd_iters, prm->svd_seed, prm->rank_ratio, k, w, st));
    CPCA_TRY(cg_setup(a, Lr, Lc, omega_r, omega_c, p, n, rr, rc, k, b, prm, w, st));
    CPCA_TRY(cg_solve(a, w, st, cg_iters, cg_res, &breakdown));
    if (breakdown) {
      set_error("cpca_decode_backward: L_aa is not positive definite (a graph component has no sampled node)");
      return CPCA_ERR_SINGULAR;
    }
  }
  const unsigned gp = std::min<unsigned>(ceil_div(int64_t(p) * kmax, 256), num_sms() * 8);
  const unsigned gn = std::min<unsigned>(ceil_div(int64_t(n) * kmax, 256), num_sms() * 8);
  assemble_side_kernel<<<gp, 256, 0, st>>>(p, k, kmax, w.pos0, w.Ut, b, w.vec[0][0], v.Uh);
  CPCA_LAUNCHED();
  assemble_side_kernel<<<gn, 256, 0, st>>>(n, k, kmax, w.pos1, w.Vt, b, w.vec[1][0], v.Vh);
  CPCA_LAUNCHED();
  colnorm_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(v.Uh, p, k, kmax, w.npart_u);
  CPCA_LAUNCHED();
  colnorm_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(v.Vh, n, k, kmax, w.npart_v);
  CPCA_LAUNCHED();
  const double scale = sqrt(double(n) * double(p) / (double(rr) * double(rc) * (1.0 - prm->delta)));
  norm_finish_kernel<<<1, 64, 0, st>>>(w.npart_u, w.npart_v, NORM_BLOCKS, k, w.s, scale, w.invu, w.invv,
                                       w.sigbuf, kmax);
  CPCA_LAUNCHED();
  CPCA_CUDA(cudaMemcpyAsync(w.Ubuf, v.Uh, sizeof(float) * size_t(p) * kmax, cudaMemcpyDeviceToDevice, st));
  CPCA_CUDA(cudaMemcpyAsync(w.Vbuf, v.Vh, sizeof(float) * size_t(n) * kmax, cudaMemcpyDeviceToDevice, st));
  scale_cols_kernel<<<gp, 256, 0, st>>>(w.Ubuf, int64_t(p) * kmax, kmax, w.invu);
  CPCA_LAUNCHED();
  scale_cols_kernel<<<gn, 256, 0, st>>>(w.Vbuf, int64_t(n) * kmax, kmax, w.invv);
  CPCA_LAUNCHED();
  // ---- held-out entries -> Ub, Vb, sigmab
  CPCA_CUDA(cudaMemsetAsync(v.Ub, 0, sizeof(float) * size_t(p) * kmax, st));
  CPCA_CUDA(cudaMemsetAsync(v.Vb, 0, sizeof(float) * size_t(n) * kmax, st));
  CPCA_CUDA(cudaMemsetAsync(v.sbar, 0, sizeof(double) * KMAX_LIMIT, st));
  if (nh > 0) {
    heldout_kernel<<<std::min<unsigned>(ceil_div(nh, 256), num_sms() * 4), 256, 0, st>>>(
        nh, h_row, h_col, h_grad, w.Ubuf, w.Vbuf, kmax, w.sigbuf, k, v.Ub, v.Vb, v.sbar);
    CPCA_LAUNCHED();
  }
  // ---- normalisation adjoint
  coldot_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(w.Ubuf, v.Ub, p, k, kmax, v.part);
  CPCA_LAUNCHED();
  sum_parts_kernel<<<1, 64, 0, st>>>(v.part, NORM_BLOCKS, v.dots_u);
  CPCA_LAUNCHED();
  coldot_partial_kernel<<<NORM_BLOCKS, 192, 0, st>>>(w.Vbuf, v.Vb, n, k, kmax, v.part);
  CPCA_LAUNCHED();
  sum_parts_kernel<<<1, 64, 0, st>>>(v.part, NORM_BLOCKS, v.dots_v);
  CPCA_LAUNCHED();
  norm_bwd_kernel<<<gp, 256, 0, st>>>(v.Ub, w.Ubuf, int64_t(p) * kmax, kmax, k, v.dots_u, w.invu);
  CPCA_LAUNCHED();
  norm_bwd_kernel<<<gn, 256, 0, st>>>(v.Vb, w.Vbuf, int64_t(n) * kmax, kmax, k, v.dots_v, w.invv);
  CPCA_LAUNCHED();
  // ---- adjoint PCG on L_aa (symmetric): Lambda = L_aa^-1 Uhb(a)
  const int m0 = p - rr, m1 = n - rc;
  if (m0 > 0) {
    gather_rhs_kernel<<<std::min<unsigned>(ceil_div(int64_t(m0) * k, 256), num_sms() * 4), 256, 0, st>>>(
        m0, k, w.abar0, v.Ub, kmax, v.rhs0);
    CPCA_LAUNCHED();
  }
  if (m1 > 0) {
    gather_rhs_kernel<<<std::min<unsigned>(ceil_div(int64_t(m1) * k, 256), num_sms() * 4), 256, 0, st>>>(
        m1, k, w.abar1, v.Vb, kmax, v.rhs1);
    CPCA_LAUNCHED();
  }
  a.s[0].rhs = v.rhs0;
  a.s[1].rhs = v.rhs1;
  CPCA_TRY(cg_solve(a, w, st, cg_iters, cg_res, &breakdown));
  if (breakdown) {
    set_error("cpca_decode_backward: adjoint PCG broke down");
    return CPCA_ERR_SINGULAR;
  }
  const CsrView lr{Lr->n, Lr->rowptr, Lr->col, Lr->val};
  const CsrView lc{Lc->n, Lc->rowptr, Lc->col, Lc->val};
  sampled_bar_kernel<<<std::min<unsigned>(ceil_div(int64_t(rr) * k, 256), num_sms() * 4), 256, 0, st>>>(
      rr, omega_r, lr, w.pos0, v.Ub, kmax, w.vec[0][0], k, v.Utb);
  CPCA_LAUNCHED();
  sampled_bar_kernel<<<std::min<unsigned>(ceil_div(int64_t(rc) * k, 256), num_sms() * 4), 256, 0, st>>>(
      rc, omega_c, lc, w.pos1, v.Vb, kmax, w.vec[1][0], k, v.Vtb);
  CPCA_LAUNCHED();
  double* oL0 = dLr ? dLr : v.dL0;
  double* oL1 = dLc ? dLc : v.dL1;
  if (dLr || dwr) {
    dl_decode_kernel<<<std::min(p, num_sms() * 8), 64, 0, st>>>(lr, w.pos0, w.vec[0][0], k, v.Uh, kmax, oL0);
    CPCA_LAUNCHED();
  }
  if (dLc || dwc) {
    dl_decode_kernel<<<std::min(n, num_sms() * 8), 64, 0, st>>>(lc, w.pos1, w.vec[1][0], k, v.Vh, kmax, oL1);
    CPCA_LAUNCHED();
  }
  // ---- SVD adjoint, A = X~ (m = rr >= n = rc) or A = X~^T
  const bool vspace = rc <= rr;
  const int mA = vspace ? rr : rc, nA = vspace ? rc : rr;
  const float* UA = vspace ? w.Ut : w.Vt;  // ld b
  const float* VA = vspace ? w.Vt : w.Ut;
  const float* UAb = vspace ? v.Utb : v.Vtb;  // ld k
  const float* VAb = vspace ? v.Vtb : v.Utb;
  auto applyA = [&](const float* in, float* out) -> cpca_status {  // out (mA x k) = A in (nA x k)
    if (!vspace) return tn_tall(Xt, ldxt, rr, rc, in, k, out, w.tn, st);
    return nn_tall(Xt, ldxt, rr, rc, in, k, out, w.tn, st);
  };
  auto applyAT = [&](const float* in, float* out) -> cpca_status {  // out (nA x k) = A^T in (mA x k)
    if (vspace) return tn_tall(Xt, ldxt, rr, rc, in, k, out, w.tn, st);
    return nn_tall(Xt, ldxt, rr, rc, in, k, out, w.tn, st);
  };
  CPCA_CUDA(cudaMemsetAsync(v.Ju, 0, sizeof(double) * k * k, st));
  CPCA_CUDA(cudaMemsetAsync(v.Jv, 0, sizeof(double) * k * k, st));
  cross_gram_kernel<<<ceil_div(mA, 64), 256, 0, st>>>(UA, b, UAb, k, mA, k, v.Ju);
  CPCA_LAUNCHED();
  cross_gram_kernel<<<ceil_div(nA, 64), 256, 0, st>>>(VA, b, VAb, k, nA, k, v.Jv);
  CPCA_LAUNCHED();
  svd_mid_kernel<<<1, 256, 0, st>>>(k, w.s, v.sbar, scale, v.Ju, v.Jv, v.Cm);
  CPCA_LAUNCHED();
  const unsigned gmk = std::min<unsigned>(ceil_div(int64_t(mA) * k, 256), num_sms() * 4);
  const unsigned gnk = std::min<unsigned>(ceil_div(int64_t(nA) * k, 256), num_sms() * 4);
  proj_sub_kernel<<<gmk, 256, 0, st>>>(mA, k, UAb, UA, b, v.Ju, v.B);
  CPCA_LAUNCHED();
  proj_sub_kernel<<<gnk, 256, 0, st>>>(nA, k, VAb, VA, b, v.Jv, v.D);
  CPCA_LAUNCHED();
  CPCA_TRY(applyAT(v.B, v.Cc));
  dim3 gg(ceil_div(nA, 32), ceil_div(nA, 32));
  gram_full_kernel<<<gg, 256, 0, st>>>(Xt, ldxt, rr, rc, vspace ? 1 : 0, v.G);
  CPCA_LAUNCHED();
  CPCA_CUDA(cudaMemsetAsync(v.flag, 0, sizeof(int), st));
  const size_t csm = sizeof(float) * size_t(nA);
  CPCA_CUDA(cudaFuncSetAttribute(shift_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(csm)));
  CPCA_PROF("dec_bwd_shift_cg", st);
  shift_cg_kernel<<<2 * k, 256, csm, st>>>(v.G, nA, k, v.Cc, v.D, w.s, VA, b, 1e-6, 4 * nA + 50, v.work,
                                            v.Yp, v.Yv, v.flag);
  CPCA_LAUNCHED();
  tcomb_kernel<<<gnk, 256, 0, st>>>(nA, k, v.Yp, v.Yv, w.s, v.T, v.F);
  CPCA_LAUNCHED();
  CPCA_TRY(applyA(v.T, v.AT));
  pcomb_kernel<<<gmk, 256, 0, st>>>(mA, k, UA, b, v.Cm, v.B, v.AT, w.s, v.P);
  CPCA_LAUNCHED();
  dim3 og(ceil_div(nA, 32), ceil_div(mA, 32));
  lowrank_out_kernel<<<og, 256, 0, st>>>(mA, nA, k, v.P, VA, b, UA, b, v.F, dXt, lddxt, vspace ? 0 : 1);
  CPCA_LAUNCHED();
  // ---- weights
  if (dwr) CPCA_TRY(laplacian_weight_grad(lr, wr, oL0, lap_type, dwr, v.deg, v.dD, st));
  if (dwc) CPCA_TRY(laplacian_weight_grad(lc, wc, oL1, lap_type, dwc, v.deg, v.dD, st));
  int flag = 0;
  CPCA_CUDA(cudaMemcpyAsync(&flag, v.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (flag & 1) {
    set_error("cpca_decode_backward: shifted Gram system not positive definite (repeated singular values?)");
    return CPCA_ERR_SINGULAR;
  }
  if (flag & 2) {
    set_error("cpca_decode_backward: shifted Gram CG did not reach its tolerance");
    return CPCA_ERR_NOT_CONVERGED;
  }
  return CPCA_OK;
}

// ------------------------------------------------- approximate decoders 2, 3
// With the full data Y and one upsampled, column-normalised basis (the
// appendix's approximate decoders 2 and 3): X = U (U^T Y) (side 0, U p x k)
// or X = (Y V) V^T (side 1, V n x k). The small factor (k x n or p x k) by a
// tall product over Y, then X by the output kernel with unit weights. Reads
// Y once and writes X once (HBM-bound; k <= 48).
__global__ void ones_kernel(double* s, int k) {
  if (threadIdx.x < k) s[threadIdx.x] = 1.0;
}

static size_t project_layout(int32_t p, int32_t n, int32_t ldb, float** W, float** scratch, double** ones,
                             void* ws) {
  Carve c(ws);
  float* w = c.take<float>(size_t(std::max(p, n)) * ldb);
  float* sc = c.take<float>(skinny_scratch_floats(p, n, ldb));
  double* o = c.take<double>(KMAX_LIMIT);
  if (W) *W = w;
  if (scratch) *scratch = sc;
  if (ones) *ones = o;
  return c.bytes();
}

extern "C" size_t cpca_subspace_project_workspace_size(int32_t p, int32_t n, int32_t ldb) {
  if (p <= 0 || n <= 0 || ldb <= 0 || ldb > KMAX_LIMIT) return 0;
  return project_layout(p, n, ldb, nullptr, nullptr, nullptr, nullptr);
}

extern "C" cpca_status cpca_subspace_project(int32_t side, const float* basis, int32_t ldb, int32_t k,
                                             const float* Y, int64_t ldy, int32_t p, int32_t n, float* X,
                                             int64_t ldx, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_subspace_project");
  CPCA_CHECK_ARG(basis && Y && X, "cpca_subspace_project: null pointer");
  CPCA_CHECK_ARG(side == 0 || side == 1, "cpca_subspace_project: side must be 0 (U) or 1 (V)");
  CPCA_CHECK_ARG(p > 0 && n > 0 && ldb >= 1 && ldb <= KMAX_LIMIT && k >= 0 && k <= ldb,
                 "cpca_subspace_project: bad sizes (p %d, n %d, ldb %d, k %d)", p, n, ldb, k);
  CPCA_CHECK_ARG(ldy >= n && ldx >= n, "cpca_subspace_project: leading dimension too small");
  float *W = nullptr, *scr = nullptr;
  double* ones = nullptr;
  const size_t need = project_layout(p, n, ldb, &W, &scr, &ones, ws);
  if (!ws || ws_bytes < need) {
    set_error("cpca_subspace_project: workspace %zu bytes < required %zu", ws_bytes, need);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (k == 0) {
    CPCA_CUDA(cudaMemset2DAsync(X, ldx * sizeof(float), 0, size_t(n) * sizeof(float), p, st));
    return CPCA_OK;
  }
  ones_kernel<<<1, 64, 0, st>>>(ones, k);
  CPCA_LAUNCHED();
  if (side == 0) {
    CPCA_PROF("project_small", st);
    CPCA_TRY(tn_tall(Y, ldy, p, n, basis, ldb, W, scr, st));  // W = Y^T U (n x ldb)
    CPCA_PROF("project_output", st);
    CPCA_TRY(launch_output(basis, ldb, W, ldb, ones, k, p, n, X, ldx, st));
  } else {
    CPCA_PROF("project_small", st);
    CPCA_TRY(nn_tall(Y, ldy, p, n, basis, ldb, W, scr, st));  // W = Y V (p x ldb)
    CPCA_PROF("project_output", st);
    CPCA_TRY(launch_output(W, ldb, basis, ldb, ones, k, p, n, X, ldx, st));
  }
  return CPCA_OK;
}

extern "C" cpca_status cpca_decode_entries(const float* U, const float* V, int32_t ld, const double* sigma,
                                           int32_t k, int64_t nh, const int32_t* h_row, const int32_t* h_col,
                                           float* out, void* stream) {
  clear_error();
  CPCA_CHECK_ARG(nh >= 0 && k >= 0 && ld >= k, "cpca_decode_entries: bad sizes");
  CPCA_CHECK_ARG(nh == 0 || (U && V && sigma && h_row && h_col && out), "cpca_decode_entries: null pointer");
  if (nh == 0) return CPCA_OK;
  entries_kernel<<<std::min<unsigned>(ceil_div(nh, 256), num_sms() * 4), 256, 0,
                   static_cast<cudaStream_t>(stream)>>>(nh, h_row, h_col, U, ld, V, ld, sigma, k, out);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

extern "C" size_t cpca_kron_reduce_workspace_size(int32_t N, int32_t rho, int64_t nnz) {
  if (N <= 0 || rho <= 0 || rho > N || nnz < 0) return 0;
  return kron_layout(nullptr, N, rho, nnz).bytes;
}

extern "C" cpca_status cpca_kron_reduce(const cpca_csr* L, const int32_t* omega, int32_t rho, double tol,
                                        int32_t max_iter, float* Lt, int64_t ldlt, int64_t* rowptr, int32_t* col,
                                        float* val, cpca_kron_info* info, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_kron_reduce");
  CPCA_CHECK_ARG(L && omega && Lt, "cpca_kron_reduce: null pointer");
  CPCA_CHECK_ARG((rowptr == nullptr) == (col == nullptr) && (col == nullptr) == (val == nullptr),
                 "cpca_kron_reduce: rowptr, col and val go together");
  const int N = L->n;
  CPCA_CHECK_ARG(N >= 1 && rho >= 1 && rho <= N, "cpca_kron_reduce: need 1 <= rho <= n (rho %d, n %d)", rho, N);
  CPCA_CHECK_ARG(ldlt >= rho, "cpca_kron_reduce: ldlt < rho");
  CPCA_CHECK_ARG(tol > 0, "cpca_kron_reduce: tol must be positive");
  CPCA_TRY(check_csr(L, N, "cpca_kron_reduce(L)"));
  const KronWs w = kron_layout(ws, N, rho, L->nnz);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_kron_reduce: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int bad = 0;
  CPCA_CUDA(cudaMemsetAsync(w.bad, 0, sizeof(int), st));
  kron_omega_check_kernel<<<std::max(1u, std::min(ceil_div(rho, 256), 64u)), 256, 0, st>>>(omega, rho, N, w.bad);
  CPCA_LAUNCHED();
  CPCA_CUDA(cudaMemcpyAsync(&bad, w.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  CPCA_CHECK_ARG(!bad, "cpca_kron_reduce: omega must be strictly ascending within [0, n)");

  const int kc = std::min(rho, KMAX_LIMIT);
  cpca_decode_params prm{};
  prm.cg_tol = tol;
  prm.cg_max_iter = max_iter;
  prm.kmax = kc;
  CgArgs a{};
  CPCA_TRY(cg_setup(a, L, L, omega, omega, 1, N, 1, rho, kc, kc, &prm, w.d, st, true, 2));
  a.s[1].R = w.R;
  a.s[1].ldr = kc;
  const CsrView lv{L->n, L->rowptr, L->col, L->val};
  int itmax = 0, chunks = 0;
  double resmax = 0.0;
  for (int j0 = 0; j0 < rho; j0 += kc) {
    const int kcur = std::min(kc, rho - j0);
    a.k = kcur;  // the PCG vectors are m x kcur for this chunk
    kron_identity_kernel<<<std::min<unsigned>(ceil_div(int64_t(rho) * kc, 256), num_sms() * 4), 256, 0, st>>>(
        w.R, rho, kc, j0, kcur);
    CPCA_LAUNCHED();
    int iters[2 * KMAX_LIMIT] = {0};
    double res[2 * KMAX_LIMIT] = {0};
    int breakdown = 0;
    CPCA_TRY(cg_solve(a, w.d, st, iters, res, &breakdown));
    if (breakdown & 2) {
      set_error("cpca_kron_reduce: a connected component holds no sampled node");
      return CPCA_ERR_SINGULAR;
    }
    for (int c = 0; c < kcur; ++c) {
      itmax = std::max(itmax, iters[KMAX_LIMIT + c]);
      resmax = std::max(resmax, res[KMAX_LIMIT + c]);
    }
    CPCA_PROF("kron_cols", st);
    kron_cols_kernel<<<std::min<unsigned>(ceil_div(int64_t(rho) * kcur, 256), num_sms() * 8), 256, 0, st>>>(
        lv, omega, w.d.pos1, w.d.vec[1][0], rho, kcur, j0, Lt, ldlt);
    CPCA_LAUNCHED();
    ++chunks;
  }
  const unsigned gsq = std::min<unsigned>(ceil_div(int64_t(rho) * rho, 256), num_sms() * 8);
  kron_sym_kernel<<<gsq, 256, 0, st>>>(Lt, ldlt, rho);
  CPCA_LAUNCHED();
  if (rowptr) {
    kron_csr_kernel<<<gsq, 256, 0, st>>>(Lt, ldlt, rho, rowptr, col, val);
    CPCA_LAUNCHED();
  }
  if (info) {
    info->chunks = chunks;
    info->cg_iters = itmax;
    info->cg_res = resmax;
  }
  if (resmax > tol) {
    set_error("cpca_kron_reduce: PCG stopped at relative residual %g", resmax);
    return CPCA_ERR_NOT_CONVERGED;
  }
  return CPCA_OK;
}
