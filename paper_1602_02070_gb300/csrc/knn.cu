// knn.cu - exact kNN graph and Laplacian (Sec. I graph construction;
// Sec. VII-A: K nearest neighbours, Gaussian kernel, sigma^2 from the
// kNN distances).
//
// Pipeline (all on the device):
//   1. candidates: tiled |a|^2 + |b|^2 - 2 a.b ranks every base point for
//      every query; each query keeps its M best per base-range split
//      (the tensor-core path in knn_tc.cu replaces this pass on sm_103a
//      when the shapes allow);
//   2. recheck: the candidates' squared distances are recomputed directly as
//      sum_t (a_t - b_t)^2 in FP32 with a fixed summation tree (so d2(i,j)
//      and d2(j,i) are bitwise equal); candidates whose order against the
//      K-th the FP32 error bound cannot settle are re-scored in FP64, so the
//      K kept are the K nearest by exact distance, ties by index; a
//      certificate checks that no point outside the candidate lists can
//      beat the K-th; queries that fail it are redone by brute force over
//      the whole grid;
//   3. graph: OR-symmetrised edge lists, sigma^2, Gaussian weights, degrees
//      and the Laplacian in CSR with sorted columns and explicit diagonal.
#include "common.cuh"
#include "knn_internal.cuh"

namespace cpca {
namespace {

constexpr int BQ = 64, BB = 64, BD = 16, KNN_THREADS = 256;

__global__ void transpose_kernel(const float* __restrict__ in, int rows, int cols, int64_t ldin,
                                 float* __restrict__ out, int64_t ldout) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[int64_t(r) * ldin + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[int64_t(c) * ldout + r] = tile[threadIdx.x][i];
  }
}

// Squared norms for candidate ranking only (FP32); also the largest norm
// (nmax_bits[0]) and the largest coordinate magnitude (nmax_bits[1]).
__global__ void norms_kernel(const float* __restrict__ P, int N, int d, int64_t ld,
                             float* __restrict__ nrm, unsigned int* __restrict__ nmax_bits) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= N) return;
  const float* a = P + int64_t(w) * ld;
  float s = 0.f, m = 0.f;
  for (int t = lane; t < d; t += 32) {
    s = fmaf(a[t], a[t], s);
    m = fmaxf(m, fabsf(a[t]));
  }
  s = warp_sumf(s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    nrm[w] = s;
    atomicMax(nmax_bits, __float_as_uint(s));  // s >= 0: bit order = value order
    atomicMax(nmax_bits + 1, __float_as_uint(m));
  }
}

// Power-of-two scale of the half-precision operand copy and the terms of
// the candidate error bound that it adds (see knn_tc_err_rel):
// sc[0] = s = 2^e with max|x| s <= 2^14 (far inside the half range),
// sc[1] = 1 / s^2 (ranking values back in the data's units),
// sc[2] = 2 a sqrt(d) and sc[3] = 2 a^2 d, a = 2^-25 / s the largest
// absolute rounding error of a coordinate that lands among the half
// subnormals. Non-finite or zero data keep s = 1.
__global__ void half_scale_kernel(const unsigned int* __restrict__ nmax_bits, int d, float* __restrict__ sc) {
  const float m = __uint_as_float(nmax_bits[1]);
  int e = 0;
  if (m > 0.f && m < __int_as_float(0x7f800000)) {
    int ex;
    (void)frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1): m < 2^ex
    e = min(max(14 - ex, -100), 100);
  }
  const double s = ldexp(1.0, e), a = ldexp(1.0, -25 - e);
  sc[0] = float(s);
  sc[1] = float(ldexp(1.0, -2 * e));
  sc[2] = float(2.0 * a * sqrt(double(d)));
  sc[3] = float(2.0 * a * a * double(d));
}

// H = half(s P), rows padded with zeros to ldh: a warp per row, lanes
// over 8-half (16-byte) groups of the row.
__global__ void __launch_bounds__(256)
to_half_kernel(const float* __restrict__ P, int N, int d, int64_t ld, const float* __restrict__ sc,
               __half* __restrict__ H, int64_t ldh) {
  const float s = sc[0];
  const int lane = threadIdx.x & 31;
  const int64_t ng = ldh / 8;  // 8-half groups per row (ldh % 8 == 0)
  const bool vec = (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(P) & 15) == 0;
  for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < N;
       i += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const float* p = P + i * ld;
    uint4* h = reinterpret_cast<uint4*>(H + i * ldh);
    for (int64_t g = lane; g < ng; g += 32) {
      const int k = int(g * 8);
      float v[8];
      if (vec && k + 8 <= d) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p + k));
        const float4 y = __ldg(reinterpret_cast<const float4*>(p + k + 4));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = k + t < d ? __ldg(p + k + t) : 0.f;
      }
      __half2 o[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) o[t] = __halves2half2(__float2half_rn(v[2 * t] * s), __float2half_rn(v[2 * t + 1] * s));
      h[g] = *reinterpret_cast<const uint4*>(o);
    }
  }
}

// Insert (d, j) into a list sorted ascending by (d, j) of length M.
template <int M>
__device__ __forceinline__ void list_insert(float* ld_, int32_t* li, float d, int32_t j) {
  if (!(d < ld_[M - 1] || (d == ld_[M - 1] && j < li[M - 1]))) return;
  int pos = M - 1;
  while (pos > 0 && (d < ld_[pos - 1] || (d == ld_[pos - 1] && j < li[pos - 1]))) {
    ld_[pos] = ld_[pos - 1];
    li[pos] = li[pos - 1];
    --pos;
  }
  ld_[pos] = d;
  li[pos] = j;
}

// Candidate pass: block (x = query tile of 64, y = split of the base range).
template <int M>
__global__ void __launch_bounds__(KNN_THREADS)
knn_candidates_kernel(const float* __restrict__ P, int N, int d, int64_t ld,
                      const float* __restrict__ nrm, int splits,
                      int32_t* __restrict__ cand_i, float* __restrict__ cand_d) {
  extern __shared__ float smem[];
  float* As = smem;                    // [BD][BQ]
  float* Bs = As + BD * BQ;            // [BD][BB]
  float* Dt = Bs + BD * BB;            // [BQ][BB+1]
  float* cd = Dt + BQ * (BB + 1);      // [BQ][M]
  int32_t* ci = reinterpret_cast<int32_t*>(cd + BQ * M);  // [BQ][M]

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int q0 = blockIdx.x * BQ;
  const int ntiles = (N + BB - 1) / BB;
  const int per = (ntiles + splits - 1) / splits;
  const int t_lo = blockIdx.y * per, t_hi = min(ntiles, t_lo + per);

  for (int e = tid; e < BQ * M; e += KNN_THREADS) {
    cd[e] = __int_as_float(0x7f800000);
    ci[e] = -1;
  }
  float nq[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = q0 + ty * 4 + i;
    nq[i] = q < N ? nrm[q] : 0.f;
  }
  const int lr = tid >> 2, lc = (tid & 3) * 4;

  for (int t = t_lo; t < t_hi; ++t) {
    const int b0 = t * BB;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += BD) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + lc + u;
        const int q = q0 + lr, b = b0 + lr;
        As[(lc + u) * BQ + lr] = (q < N && k < d) ? P[int64_t(q) * ld + k] : 0.f;
        Bs[(lc + u) * BB + lr] = (b < N && k < d) ? P[int64_t(b) * ld + k] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BD; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(As + k * BQ + ty * 4);
        const float4 b = *reinterpret_cast<const float4*>(Bs + k * BB + tx * 4);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = q0 + ty * 4 + i, b = b0 + tx * 4 + j;
        float v = __int_as_float(0x7f800000);
        if (b < N && b != q) v = nq[i] + nrm[b] - 2.f * acc[i][j];
        Dt[(ty * 4 + i) * (BB + 1) + tx * 4 + j] = v;
      }
    __syncthreads();
    if (tid < BQ) {
      float* myd = cd + tid * M;
      int32_t* myi = ci + tid * M;
      const float* row = Dt + tid * (BB + 1);
      for (int j = 0; j < BB; ++j) {
        const float v = row[j];
        if (v <= myd[M - 1]) list_insert<M>(myd, myi, v, b0 + j);
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < BQ * M; e += KNN_THREADS) {
    const int q = q0 + e / M;
    if (q < N) {
      const int64_t o = (int64_t(blockIdx.y) * N + q) * M + (e % M);
      cand_i[o] = ci[e];
      cand_d[o] = cd[e];
    }
  }
}

}  // namespace

// Exact squared distance, FP32, fixed summation tree: lane l sums
// coordinates l, l+32, ... (or float4 groups), then a butterfly; lane 0's
// value is broadcast. (a-b)^2 == (b-a)^2, so d2(i,j) == d2(j,i) bitwise.
__device__ __forceinline__ float exact_d2_warp(const float* __restrict__ a,
                                               const float* __restrict__ b, int d, bool vec4) {
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  if (vec4) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (int t = lane; t < (d >> 2); t += 32) {
      const float4 x = __ldg(a4 + t), y = __ldg(b4 + t);
      float dx = x.x - y.x;
      s = fmaf(dx, dx, s);
      dx = x.y - y.y;
      s = fmaf(dx, dx, s);
      dx = x.z - y.z;
      s = fmaf(dx, dx, s);
      dx = x.w - y.w;
      s = fmaf(dx, dx, s);
    }
  } else {
    for (int t = lane; t < d; t += 32) {
      const float dx = __ldg(a + t) - __ldg(b + t);
      s = fmaf(dx, dx, s);
    }
  }
  s = warp_sumf(s);
  return __shfl_sync(0xffffffffu, s, 0);
}

// exact_d2_warp from one point a to up to G points (row c[g] of P for
// g < n), each with exactly exact_d2_warp's arithmetic, a's coordinates read
// once for all of them.
template <int G>
__device__ __forceinline__ void exact_d2_warp_group(const float* __restrict__ a, const float* __restrict__ P,
                                                    int64_t ld, const int* c, int n, int d, bool vec4,
                                                    float* out) {
  const int lane = threadIdx.x & 31;
  float s[G];
  const float* b[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    s[g] = 0.f;
    b[g] = P + int64_t(g < n ? c[g] : c[0]) * ld;
  }
  if (vec4) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    for (int t = lane; t < (d >> 2); t += 32) {
      const float4 x = __ldg(a4 + t);
      float4 y[G];
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < n) y[g] = __ldg(reinterpret_cast<const float4*>(b[g]) + t);
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < n) {
          float dx = x.x - y[g].x;
          s[g] = fmaf(dx, dx, s[g]);
          dx = x.y - y[g].y;
          s[g] = fmaf(dx, dx, s[g]);
          dx = x.z - y[g].z;
          s[g] = fmaf(dx, dx, s[g]);
          dx = x.w - y[g].w;
          s[g] = fmaf(dx, dx, s[g]);
        }
    }
  } else {
    for (int t = lane; t < d; t += 32) {
      const float x = __ldg(a + t);
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < n) {
          const float dx = x - __ldg(b[g] + t);
          s[g] = fmaf(dx, dx, s[g]);
        }
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const float v = warp_sumf(s[g]);
    out[g] = __shfl_sync(0xffffffffu, v, 0);
  }
}

// The same distance in FP64 (direct differences of the FP32 inputs, which
// are exact in FP64; lane-strided FP64 sums, then a butterfly): relative
// error about (d/32 + 5) 2^-53, used only to order candidates that the FP32
// value cannot separate.
__device__ __forceinline__ double exact_d2_warp_f64(const float* __restrict__ a,
                                                    const float* __restrict__ b, int d, bool vec4) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (vec4) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (int t = lane; t < (d >> 2); t += 32) {
      const float4 x = __ldg(a4 + t), y = __ldg(b4 + t);
      double dx = double(x.x) - double(y.x);
      s = fma(dx, dx, s);
      dx = double(x.y) - double(y.y);
      s = fma(dx, dx, s);
      dx = double(x.z) - double(y.z);
      s = fma(dx, dx, s);
      dx = double(x.w) - double(y.w);
      s = fma(dx, dx, s);
    }
  } else {
    for (int t = lane; t < d; t += 32) {
      const double dx = double(__ldg(a + t)) - double(__ldg(b + t));
      s = fma(dx, dx, s);
    }
  }
  s = warp_sum(s);
  return __shfl_sync(0xffffffffu, s, 0);
}

// Relative error bound of exact_d2_warp: each lane adds about d/32 rounded
// squares of rounded differences in order (2 + d/32 roundings), then a
// five-level butterfly; 16 covers the constant terms with margin.
__host__ __device__ inline float exact_d2_tau(int d) { return float((d / 32.0 + 16.0) * 0x1.0p-24); }

namespace {

constexpr int RECHECK_WARPS = 4;
constexpr int kRecheckGroup = 8;  // candidates scored together

// The K nearest of a warp's candidate set by exact distance. Candidate c
// (c < C) is live when si[c] >= 0 and has the FP32 exact distance sd[c],
// whose relative error is at most tau. With a_K the K-th smallest FP32
// value, a candidate below a_K (1 - tau)/(1 + tau) is certainly among the K
// nearest and one above a_K (1 + tau)/(1 - tau) certainly is not; the
// candidates in between are re-scored in FP64 (s64) and the free places go
// to the smallest of those, ties by index. Writes out_i/out_d (the FP32
// distances, symmetric in i and j), consumes si (picked entries set to -1)
// and returns the largest upper bound sd (1 + tau) of the chosen distances
// (INF when fewer than K candidates are live).
__device__ float resolve_knn(const float* __restrict__ P, int64_t ld, int d, bool vec4, int q, int K,
                             int C, const float* sd, int32_t* si, double* s64, float tau,
                             int32_t* __restrict__ out_i, float* __restrict__ out_d) {
  const int lane = threadIdx.x & 31;
  const float INF = __int_as_float(0x7f800000);
  // a_K: K rounds of a warp argmin over (sd, index)
  float aK = INF;
  for (int r = 0; r < K; ++r) {
    float bd = INF;
    int bj = 0x7fffffff, bc = -1;
    for (int c = lane; c < C; c += 32) {
      const int j = si[c];
      if (j < 0) continue;
      const float v = sd[c];
      if (v < bd || (v == bd && j < bj)) {
        bd = v;
        bj = j;
        bc = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (od < bd || (od == bd && oj < bj)) {
        bd = od;
        bj = oj;
        bc = oc;
      }
    }
    aK = bd;
    if (lane == 0 && bc >= 0) si[bc] = -2 - si[bc];  // hide the pick for the next round
    __syncwarp();
  }
  for (int c = lane; c < C; c += 32)
    if (si[c] <= -2) si[c] = -2 - si[c];
  __syncwarp();
  // classes: 0 certainly in, 1 undecided (FP64), 2 certainly out
  const double lo = aK < INF ? double(aK) * (1.0 - tau) / (1.0 + tau) : double(INF);
  const double hi = aK < INF ? double(aK) * (1.0 + tau) / (1.0 - tau) : double(INF);
  for (int c = 0; c < C; ++c) {
    const int j = si[c];
    if (j < 0 || aK == INF) continue;  // warp-uniform
    const double v = double(sd[c]);
    if (v >= lo && v <= hi) {
      const double w = exact_d2_warp_f64(P + int64_t(q) * ld, P + int64_t(j) * ld, d, vec4);
      if (lane == 0) s64[c] = w;
    }
  }
  __syncwarp();
  float up = 0.f;
  for (int r = 0; r < K; ++r) {
    int bk = 3;  // class
    double bv = 0.0;
    int bj = 0x7fffffff, bc = -1;
    for (int c = lane; c < C; c += 32) {
      const int j = si[c];
      if (j < 0) continue;
      const double v32 = double(sd[c]);
      const int k = (aK == INF || v32 < lo) ? 0 : (v32 <= hi ? 1 : 2);
      if (k == 2) continue;
      const double v = k == 0 ? v32 : s64[c];
      if (k < bk || (k == bk && (v < bv || (v == bv && j < bj)))) {
        bk = k;
        bv = v;
        bj = j;
        bc = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ok < bk || (ok == bk && (ov < bv || (ov == bv && oj < bj)))) {
        bk = ok;
        bv = ov;
        bj = oj;
        bc = oc;
      }
    }
    const float dv = bc >= 0 ? sd[bc] : INF;
    if (lane == 0) {
      out_i[int64_t(q) * K + r] = bc >= 0 ? bj : 0x7fffffff;
      out_d[int64_t(q) * K + r] = dv;
      if (bc >= 0) si[bc] = -1;
    }
    up = fmaxf(up, dv * (1.f + tau));
    __syncwarp();
  }
  return up;
}

// Recheck: warp per query. With e = err_rel (|q|^2 + max |b|^2) (plus, for
// the half-precision candidates, err_abs[0] (|q| + max |b|) + err_abs[1])
// bounding |ranking value - exact squared distance|, let a_K be the K-th smallest
// ranking value over all candidates. A candidate whose ranking value
// exceeds a_K + 2e has exact distance > a_K + e, while the K candidates at
// or below a_K have exact distance <= a_K + e, so it cannot be among the K
// nearest: only the candidates within a_K + 2e are re-scored exactly
// (FP32, and FP64 where FP32 cannot decide: resolve_knn). Then the
// certificate is evaluated.
__global__ void __launch_bounds__(RECHECK_WARPS * 32)
knn_recheck_kernel(const float* __restrict__ P, int N, int d, int64_t ld, bool vec4, int K,
                   int M, int splits, const int32_t* __restrict__ cand_i,
                   const float* __restrict__ cand_d, const float* __restrict__ nrm,
                   const unsigned int* __restrict__ nmax_bits, float err_rel,
                   const float* __restrict__ err_abs, int32_t* __restrict__ out_i, float* __restrict__ out_d,
                   int32_t* __restrict__ redo, int32_t* __restrict__ n_redo) {
  extern __shared__ double smd[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = splits * M;
  double* s64 = smd + size_t(wib) * C;                              // FP64 distances
  float* sa = reinterpret_cast<float*>(smd + size_t(RECHECK_WARPS) * C) + size_t(wib) * C * 3;  // ranking values
  float* sd = sa + C;                                     // exact squared distances
  int32_t* si = reinterpret_cast<int32_t*>(sd + C);       // candidate indices
  const int q = blockIdx.x * RECHECK_WARPS + wib;
  if (q >= N) return;
  const float INF = __int_as_float(0x7f800000);
  const float nbmax = __uint_as_float(*nmax_bits);
  float e = err_rel * (nrm[q] + nbmax);
  if (err_abs) e += err_abs[0] * (sqrtf(nrm[q]) + sqrtf(nbmax)) + err_abs[1];
  for (int c = lane; c < C; c += 32) {
    const int s = c / M, m = c % M;
    const int64_t o = (int64_t(s) * N + q) * M + m;
    const int j = cand_i[o];
    si[c] = j;
    const float a = cand_d[o];
    sa[c] = j >= 0 && a == a ? a : INF;
    sd[c] = INF;
  }
  __syncwarp();
  // a_K: K rounds of a warp argmin over the ranking values (continued to
  // a_2K, the 2K-th, for the case below)
  float aK = INF, a2K = INF;
  for (int r = 0; r < 2 * K; ++r) {
    float bv = INF;
    int bc = -1;
    for (int c = lane; c < C; c += 32) {
      const float v = sa[c];
      if (si[c] >= 0 && v < bv) {
        bv = v;
        bc = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ov < bv || (ov == bv && oc >= 0 && (bc < 0 || oc < bc))) {
        bv = ov;
        bc = oc;
      }
    }
    if (r < K) aK = bv;
    a2K = bv;
    if (lane == 0 && bc >= 0) si[bc] = -2 - si[bc];  // temporarily hide the pick
    __syncwarp();
  }
  for (int c = lane; c < C; c += 32)
    if (si[c] <= -2) si[c] = -2 - si[c];
  __syncwarp();
  float window = aK + 2.f * e;
  // Such a query is not certified: it is searched by brute force within the
  // budget, else left uncertified, and its exact re-scoring is kept to the
  // 2K best ranking values (the ranking error in practice is far below the
  // gaps that separate them from the K-th).
  // A full split list whose last ranking value lies within a_K + e leaves
  // room for a point beyond it as close as the K-th: the certificate is not
  // attempted (the query goes to the brute-force budget)
  bool hopeless = false;
  for (int s = 0; s < splits; ++s) {
    const int64_t o = (int64_t(s) * N + q) * M + (M - 1);
    if (cand_i[o] >= 0 && cand_d[o] <= aK + e) hopeless = true;
  }
  if (hopeless) window = fminf(window, a2K);
  // the candidates within the window, scored eight at a time (the query's
  // coordinates read once per group)
  __shared__ int grp[RECHECK_WARPS][kRecheckGroup];
  __shared__ int grj[RECHECK_WARPS][kRecheckGroup];
  int n = 0;
  auto flush = [&]() {
    float v[kRecheckGroup];
    exact_d2_warp_group<kRecheckGroup>(P + int64_t(q) * ld, P, ld, grj[wib], n, d, vec4, v);
    if (lane == 0)
      for (int g = 0; g < n; ++g) sd[grp[wib][g]] = v[g] != v[g] ? INF : v[g];  // NaN input ranks last
    __syncwarp();
  };
  for (int c = 0; c < C; ++c) {
    const int j = si[c];
    if (j < 0) continue;
    __syncwarp();
    if (!(sa[c] <= window)) {  // warp-uniform branch: never among the K nearest
      if (lane == 0) si[c] = -1;
      __syncwarp();
      continue;
    }
    if (lane == 0) {
      grp[wib][n] = c;
      grj[wib][n] = j;
    }
    __syncwarp();
    if (++n == kRecheckGroup) {
      flush();
      n = 0;
    }
  }
  if (n > 0) flush();
  __syncwarp();
  const float dK = resolve_knn(P, ld, d, vec4, q, K, C, sd, si, s64, exact_d2_tau(d), out_i, out_d);
  // Certificate: every point outside split s's list has a ranking value
  // >= that list's last entry, hence an exact distance >= that minus e,
  // which must exceed every chosen exact distance (at most dK).
  if (lane == 0) {
    bool ok = dK < INF && !hopeless;
    for (int s = 0; s < splits; ++s) {
      const float thr = cand_d[(int64_t(s) * N + q) * M + (M - 1)];
      if (!(thr - e > dK)) {
        if (cand_i[(int64_t(s) * N + q) * M + (M - 1)] >= 0) ok = false;  // full list
      }
    }
    if (!ok) redo[atomicAdd(n_redo, 1)] = q;
  }
}

// Brute force for queries without a certificate, spread over the grid.
// Work item (r, c): redo query r of the batch [r0, r0 + nq) against points
// [c * chunk, (c + 1) * chunk), one warp per item, every point scored
// with the same exact FP32 function; the warp keeps the 32 nearest by
// (d2, j) (lane l holds entry l, insertion by ballot) and writes them to
// lists[r][c]. knn_bf_merge_kernel then takes, per query, the 32 nearest of
// all its chunk lists and lets resolve_knn pick the K (FP64 where FP32 cannot
// decide; a tie run longer than the 32 kept is cut at the 32nd).
constexpr int kBfChunkMin = 32, kBfChunkMax = 512;  // points per work item
constexpr int kBfBatch = 64;  // queries per brute-force pass

__device__ __forceinline__ void warp_list_insert(float& ld_, int& li, float v, int j) {
  const int lane = threadIdx.x & 31;
  const float last = __shfl_sync(0xffffffffu, ld_, 31);
  const int lastj = __shfl_sync(0xffffffffu, li, 31);
  if (!(lastj < 0 || v < last || (v == last && j < lastj))) return;  // warp-uniform
  const bool before = li >= 0 && (ld_ < v || (ld_ == v && li < j));
  const int pos = __popc(__ballot_sync(0xffffffffu, before));
  const float up = __shfl_up_sync(0xffffffffu, ld_, 1);
  const int upj = __shfl_up_sync(0xffffffffu, li, 1);
  if (lane > pos) {
    ld_ = up;
    li = upj;
  } else if (lane == pos) {
    ld_ = v;
    li = j;
  }
}

__global__ void __launch_bounds__(RECHECK_WARPS * 32)
knn_bf_score_kernel(const float* __restrict__ P, int N, int d, int64_t ld, bool vec4,
                    const int32_t* __restrict__ redo, int r0, int nq, int chunk, float* __restrict__ lists_d,
                    int32_t* __restrict__ lists_i) {
  const int lane = threadIdx.x & 31;
  const int nch = (N + chunk - 1) / chunk;
  const int64_t items = int64_t(nq) * nch;
  for (int64_t w = int64_t(blockIdx.x) * RECHECK_WARPS + (threadIdx.x >> 5); w < items;
       w += int64_t(gridDim.x) * RECHECK_WARPS) {
    const int r = int(w / nch), c = int(w % nch);
    const int q = redo[r0 + r];
    const float* a = P + int64_t(q) * ld;
    float dl = __int_as_float(0x7f800000);
    int il = -1;
    const int j1 = min(N, (c + 1) * chunk);
    for (int j0 = c * chunk; j0 < j1; j0 += kRecheckGroup) {  // eight points per pass
      const int n = min(kRecheckGroup, j1 - j0);
      int jj[kRecheckGroup];
#pragma unroll
      for (int g = 0; g < kRecheckGroup; ++g) jj[g] = j0 + min(g, n - 1);
      float v[kRecheckGroup];
      exact_d2_warp_group<kRecheckGroup>(a, P, ld, jj, n, d, vec4, v);
#pragma unroll
      for (int g = 0; g < kRecheckGroup; ++g) {
        if (g >= n || j0 + g == q) continue;  // warp-uniform
        warp_list_insert(dl, il, v[g] != v[g] ? __int_as_float(0x7f800000) : v[g], j0 + g);
      }
    }
    lists_d[w * 32 + lane] = dl;
    lists_i[w * 32 + lane] = il;
  }
}

__global__ void __launch_bounds__(RECHECK_WARPS * 32)
knn_bf_merge_kernel(const float* __restrict__ P, int N, int d, int64_t ld, bool vec4, int K,
                    const int32_t* __restrict__ redo, int r0, int nq, int chunk, const float* __restrict__ lists_d,
                    const int32_t* __restrict__ lists_i, int32_t* __restrict__ out_i,
                    float* __restrict__ out_d) {
  __shared__ double l64[RECHECK_WARPS][32];
  __shared__ float sd[RECHECK_WARPS][32];
  __shared__ int32_t si[RECHECK_WARPS][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * RECHECK_WARPS + wib;
  if (r >= nq) return;
  const int q = redo[r0 + r];
  const int nch = (N + chunk - 1) / chunk;
  float dl = __int_as_float(0x7f800000);
  int il = -1;
  for (int c = 0; c < nch; ++c) {
    const int64_t o = (int64_t(r) * nch + c) * 32;
    const float vd = lists_d[o + lane];
    const int vi = lists_i[o + lane];
    for (int t = 0; t < 32; ++t) {  // entries in list order (ascending)
      const float v = __shfl_sync(0xffffffffu, vd, t);
      const int j = __shfl_sync(0xffffffffu, vi, t);
      if (j < 0) break;  // warp-uniform: the rest of the list is empty
      warp_list_insert(dl, il, v, j);
    }
  }
  sd[wib][lane] = dl;
  si[wib][lane] = il;
  __syncwarp();
  resolve_knn(P, ld, d, vec4, q, K, min(32, N - 1), sd[wib], si[wib], l64[wib], exact_d2_tau(d), out_i, out_d);
}

// ------------------------------------------------------------ graph build --
constexpr int RED_BLOCKS = 256;

// Deterministic FP64 sum of an FP32 array: fixed block partials, then one
// block adds the partials in order.
__global__ void sum_partials_kernel(const float* __restrict__ x, int64_t m, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m;
       t += int64_t(gridDim.x) * blockDim.x)
    s += double(x[t]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void sigma2_finish_kernel(const double* __restrict__ part, int nparts, int64_t m,
                                     double given, double* __restrict__ sigma2) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (given > 0) {
      *sigma2 = given;
    } else {
      double s = 0.0;
      for (int i = 0; i < nparts; ++i) s += part[i];
      *sigma2 = s / double(m);
    }
  }
}

__global__ void indeg_kernel(const int32_t* __restrict__ knn, int N, int K, int32_t* __restrict__ indeg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(N) * K;
       t += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(&indeg[knn[t]], 1);
}

// Single-block exclusive scan of (base + add[i]) into out[0..N] (int64).
__global__ void scan_kernel(const int32_t* __restrict__ add, int base, int N, int64_t* __restrict__ out) {
  __shared__ int64_t sh[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int chunk = (N + nt - 1) / nt;
  const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
  int64_t s = 0;
  for (int i = lo; i < hi; ++i) s += base + add[i];
  sh[tid] = s;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    int64_t v = tid >= o ? sh[tid - o] : 0;
    __syncthreads();
    sh[tid] += v;
    __syncthreads();
  }
  int64_t run = sh[tid] - s;
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    run += base + add[i];
  }
  if (tid == nt - 1) out[N] = sh[nt - 1];
}

__global__ void fill_edges_kernel(const int32_t* __restrict__ knn, const float* __restrict__ kd2, int N,
                                  int K, const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                                  int32_t* __restrict__ e_nbr, float* __restrict__ e_d2) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(N) * K;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / K), k = int(t % K);
    const int j = knn[t];
    const float v = kd2[t];
    e_nbr[off[i] + k] = j;
    e_d2[off[i] + k] = v;
    const int64_t slot = off[j] + K + atomicAdd(&cursor[j], 1);
    e_nbr[slot] = i;
    e_d2[slot] = v;
  }
}

// Per node: sort its edge list by neighbour, drop duplicates (an edge seen
// from both ends carries the same bitwise d2), count what is left.
// Sort each node's edge list by neighbour and drop repeats (an edge listed
// by both ends), in place. A warp per node: every entry's rank among the
// distinct neighbours comes from comparisons with all entries (shuffles),
// then the kept entries are written at their ranks. The first copy of a
// repeat is kept (repeats carry the same squared distance anyway: it is
// symmetric bit for bit). Lists longer than kDedupeWarpMax (hub nodes of a
// kNN graph in high dimension) are queued for dedupe_long_kernel.
constexpr int kDedupeSlots = 8, kDedupeWarpMax = 32 * kDedupeSlots;
constexpr int kDedupeBlockMax = 8192;  // entries one block sorts in shared memory
__global__ void __launch_bounds__(256)
dedupe_kernel(int N, const int64_t* __restrict__ off, int32_t* __restrict__ e_nbr, float* __restrict__ e_d2,
              int32_t* __restrict__ uniq, int32_t* __restrict__ longq, int32_t* __restrict__ n_long) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += (gridDim.x * blockDim.x) >> 5) {
    const int64_t lo = off[i], hi = off[i + 1];
    const int n = int(hi - lo);
    if (n > kDedupeWarpMax) {  // warp-uniform
      if (lane == 0) longq[atomicAdd(n_long, 1)] = i;
      continue;
    }
    int nb[kDedupeSlots];
    float dv[kDedupeSlots];
    bool keep[kDedupeSlots];
    int rk[kDedupeSlots];
#pragma unroll
    for (int q = 0; q < kDedupeSlots; ++q) {
      const int e = lane + 32 * q;
      nb[q] = e < n ? e_nbr[lo + e] : 0x7fffffff;
      dv[q] = e < n ? e_d2[lo + e] : 0.f;
      keep[q] = e < n;
      rk[q] = 0;
    }
    // pass 1: an entry is a repeat when an earlier entry has its neighbour
#pragma unroll
    for (int t = 0; t < kDedupeSlots; ++t) {
      if (32 * t >= n) break;  // warp-uniform
      for (int l = 0; l < 32; ++l) {
        const int a = l + 32 * t;
        const int v = __shfl_sync(0xffffffffu, nb[t], l);
        if (a >= n) break;  // warp-uniform
#pragma unroll
        for (int q = 0; q < kDedupeSlots; ++q)
          if (v == nb[q] && a < lane + 32 * q) keep[q] = false;
      }
    }
    // pass 2: the rank of a kept entry = the kept entries with a smaller neighbour
#pragma unroll
    for (int t = 0; t < kDedupeSlots; ++t) {
      if (32 * t >= n) break;
      for (int l = 0; l < 32; ++l) {
        const int a = l + 32 * t;
        const int v = __shfl_sync(0xffffffffu, nb[t], l);
        const bool k = __shfl_sync(0xffffffffu, keep[t], l);
        if (a >= n) break;
#pragma unroll
        for (int q = 0; q < kDedupeSlots; ++q) rk[q] += (k && v < nb[q]) ? 1 : 0;
      }
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < kDedupeSlots; ++q) cnt += keep[q] ? 1 : 0;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    __syncwarp();  // every read of the list is done
#pragma unroll
    for (int q = 0; q < kDedupeSlots; ++q)
      if (keep[q]) {
        e_nbr[lo + rk[q]] = nb[q];
        e_d2[lo + rk[q]] = dv[q];
      }
    if (lane == 0) uniq[i] = cnt;
    __syncwarp();
  }
}

// The queued long lists: a block per list, keys (neighbour, position) sorted
// in shared memory by a bitonic network, then the first copy of each
// neighbour kept in order (what the warp path computes). Lists beyond
// kDedupeBlockMax entries take one thread's insertion sort.
__global__ void __launch_bounds__(1024)
dedupe_long_kernel(const int64_t* __restrict__ off, int32_t* __restrict__ e_nbr, float* __restrict__ e_d2,
                   int32_t* __restrict__ uniq, const int32_t* __restrict__ longq,
                   const int32_t* __restrict__ n_long) {
  extern __shared__ unsigned long long dkeys[];
  float* dval = reinterpret_cast<float*>(dkeys + kDedupeBlockMax);
  const int nl = *n_long;
  for (int t = blockIdx.x; t < nl; t += gridDim.x) {
    const int i = longq[t];
    const int64_t lo = off[i], hi = off[i + 1];
    const int n = int(hi - lo);
    if (n > kDedupeBlockMax) {  // block-uniform
      if (threadIdx.x == 0) {
        for (int64_t a = lo + 1; a < hi; ++a) {
          const int32_t j = e_nbr[a];
          const float v = e_d2[a];
          int64_t b = a;
          while (b > lo && e_nbr[b - 1] > j) {
            e_nbr[b] = e_nbr[b - 1];
            e_d2[b] = e_d2[b - 1];
            --b;
          }
          e_nbr[b] = j;
          e_d2[b] = v;
        }
        int64_t w = lo;
        for (int64_t a = lo; a < hi; ++a) {
          if (a > lo && e_nbr[a] == e_nbr[w - 1]) continue;
          e_nbr[w] = e_nbr[a];
          e_d2[w] = e_d2[a];
          ++w;
        }
        uniq[i] = int32_t(w - lo);
      }
      __syncthreads();
      continue;
    }
    int np = 1;
    while (np < n) np <<= 1;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      dkeys[e] = e < n ? (static_cast<unsigned long long>(static_cast<uint32_t>(e_nbr[lo + e])) << 32) |
                             static_cast<unsigned long long>(e)
                       : ~0ull;
      if (e < n) dval[e] = e_d2[lo + e];
    }
    __syncthreads();
    for (int k = 2; k <= np; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
          const int pe = e ^ j;
          if (pe > e) {
            const bool up = (e & k) == 0;
            const unsigned long long x = dkeys[e], y = dkeys[pe];
            if ((x > y) == up) {
              dkeys[e] = y;
              dkeys[pe] = x;
            }
          }
        }
        __syncthreads();
      }
    // keep the first (lowest position) copy of each neighbour, in order
    if (threadIdx.x == 0) {
      int w = 0;
      for (int e = 0; e < n; ++e) {
        const int32_t j = int32_t(dkeys[e] >> 32);
        if (e > 0 && j == int32_t(dkeys[e - 1] >> 32)) continue;
        const int pos = int(dkeys[e] & 0xffffffffull);
        e_nbr[lo + w] = j;
        e_d2[lo + w] = dval[pos];
        ++w;
      }
      uniq[i] = w;
    }
    __syncthreads();
  }
}

__global__ void degree_kernel(int N, const int64_t* __restrict__ off, const int32_t* __restrict__ uniq,
                              const float* __restrict__ e_d2, const double* __restrict__ sigma2,
                              double* __restrict__ deg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s2 = *sigma2;
  double D = 0.0;
  for (int64_t a = off[i]; a < off[i] + uniq[i]; ++a) D += exp(-double(e_d2[a]) / s2);
  deg[i] = D;
}

__global__ void assemble_kernel(int N, int lap_type, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ uniq, const int32_t* __restrict__ e_nbr,
                                const float* __restrict__ e_d2, const double* __restrict__ sigma2,
                                const double* __restrict__ deg, const int64_t* __restrict__ rowptr,
                                int64_t nnz_cap, int32_t* __restrict__ col, float* __restrict__ val,
                                float* __restrict__ weight) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (rowptr[N] > nnz_cap) return;  // reported by the host
  const double s2 = *sigma2;
  const double Di = deg[i];
  int64_t w = rowptr[i];
  bool diag_done = false;
  const int64_t lo = off[i], hi = off[i] + uniq[i];
  for (int64_t a = lo; a <= hi; ++a) {
    const bool at_end = a == hi;
    const int32_t j = at_end ? 0x7fffffff : e_nbr[a];
    if (!diag_done && j > i) {
      col[w] = i;
      val[w] = lap_type == CPCA_LAP_COMBINATORIAL ? float(Di) : (Di > 0 ? 1.f : 0.f);
      if (weight) weight[w] = 0.f;
      ++w;
      diag_done = true;
    }
    if (at_end) break;
    const double Wij = exp(-double(e_d2[a]) / s2);
    col[w] = j;
    if (lap_type == CPCA_LAP_COMBINATORIAL) {
      val[w] = float(-Wij);
    } else {
      const double Dj = deg[j];
      val[w] = (Di > 0 && Dj > 0) ? float(-Wij / sqrt(Di * Dj)) : 0.f;
    }
    if (weight) weight[w] = float(Wij);
    ++w;
  }
}

}  // namespace

// Layout of the kNN workspace; shared by the size query and the call.
struct KnnWs {
  float* Pt;          // transposed points (transposed input only)
  float* nrm;
  unsigned int* nmax;  // [largest squared norm, largest |coordinate|] (float bits)
  __half* H;           // half-precision operand copy for the tensor-core pass
  float* hsc;          // its scale and error terms (half_scale_kernel)
  int32_t* cand_i;
  float* cand_d;
  int32_t* kidx;      // N*K (used when the caller passes no knn_idx)
  float* kd2;
  int32_t* redo;
  int32_t* n_redo;
  float* bf_d;        // brute-force chunk lists [kBfBatch][chunks][32]
  int32_t* bf_i;
  int* err;
  double* part;
  double* sigma2;
  int32_t* indeg;
  int32_t* cursor;
  int64_t* off;
  int32_t* e_nbr;
  float* e_d2;
  int32_t* uniq;
  int32_t* longq;     // nodes whose lists dedupe_long_kernel sorts
  int32_t* n_long;
  double* deg;
  size_t bytes;
};

// Base-range splits S (each query keeps M candidates per split): the S in
// {1, 2, 4, 8} whose blocks fill the GPU in the fewest waves per unit of
// work, ceil(tiles S / SMs) / S, with 128-query tiles in pairs (the
// tensor-core pass's clusters) and at least 4 base tiles of 256 per split.
static int knn_splits(int N, int d) {
  (void)d;
  const int qt = (int(ceil_div(N, 128)) + 1) / 2 * 2;
  const int P = num_sms();
  int best = 1;
  double cost = 1e300;
  for (int s = 1; s <= 8; s *= 2) {
    if (s > 1 && (N + 255) / 256 < 4 * s) break;
    const double c = double(ceil_div(int64_t(qt) * s, P)) / s;
    if (c < cost - 1e-9) {
      cost = c;
      best = s;
    }
  }
  return best;
}

// Brute-force budget of one graph: a query costs N d FMAs; at most
// max(64, 2e11 / (N d)) uncertified queries are redone, else none is.
static int knn_bruteforce_cap(int N, int d) {
  return int(std::max<double>(64.0, std::min<double>(N, 2e11 / (double(N) * double(d)))));
}
static int knn_M(int K) { return K <= 16 ? 32 : 64; }

static KnnWs knn_layout(void* ws, int N, int d, int K, int transposed) {
  Carve c(ws);
  KnnWs w{};
  const int S = knn_splits(N, d), M = knn_M(K);
  w.Pt = transposed ? c.take<float>(size_t(N) * ((d + 3) & ~3)) : nullptr;
  w.nrm = c.take<float>(N);
  w.nmax = c.take<unsigned int>(2);
  w.H = c.take<__half>(size_t(N) * knn_half_ld(d));
  w.hsc = c.take<float>(4);
  w.cand_i = c.take<int32_t>(size_t(S) * N * M);
  w.cand_d = c.take<float>(size_t(S) * N * M);
  w.kidx = c.take<int32_t>(size_t(N) * K);
  w.kd2 = c.take<float>(size_t(N) * K);
  w.redo = c.take<int32_t>(N);
  w.n_redo = c.take<int32_t>(1);
  {
    const size_t lists = size_t(kBfBatch) * ((N + kBfChunkMin - 1) / kBfChunkMin) * 32;
    w.bf_d = c.take<float>(lists);
    w.bf_i = c.take<int32_t>(lists);
  }
  w.err = c.take<int>(1);
  w.part = c.take<double>(RED_BLOCKS);
  w.sigma2 = c.take<double>(1);
  w.indeg = c.take<int32_t>(N);
  w.cursor = c.take<int32_t>(N);
  w.off = c.take<int64_t>(size_t(N) + 1);
  w.e_nbr = c.take<int32_t>(size_t(2) * N * K);
  w.e_d2 = c.take<float>(size_t(2) * N * K);
  w.uniq = c.take<int32_t>(N);
  w.longq = c.take<int32_t>(N);
  w.n_long = c.take<int32_t>(1);
  w.deg = c.take<double>(N);
  w.bytes = c.bytes();
  return w;
}

// kNN lists (idx, d2) of points P (N x d, row stride ld, K-major) into
// out_i/out_d; P must be 16-byte aligned with ld % 4 == 0 for vector loads.
cpca_status knn_lists(const float* P, int N, int d, int64_t ld, int K, const KnnWs& w,
                      int32_t* out_i, float* out_d, int* n_bruteforce, int* n_uncertified,
                      float* err_rel_used, cudaStream_t st) {
  const int S = knn_splits(N, d), M = knn_M(K);
  const bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
  CPCA_CUDA(cudaMemsetAsync(w.nmax, 0, 2 * sizeof(unsigned int), st));
  CPCA_CUDA(cudaMemsetAsync(w.n_redo, 0, sizeof(int32_t), st));
  CPCA_PROF("knn_norms", st);
  norms_kernel<<<ceil_div(int64_t(N) * 32, 256), 256, 0, st>>>(P, N, d, ld, w.nrm, w.nmax);
  CPCA_LAUNCHED();
  bool done = false;
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  if (knn_tc_supported(N, d, M)) {
    // the operands in half precision (the same 11-bit significand as TF32,
    // twice its tensor rate): a power-of-two scale, then the copy
    half_scale_kernel<<<1, 1, 0, st>>>(w.nmax, d, w.hsc);
    CPCA_LAUNCHED();
    const int64_t ldh = knn_half_ld(d);
    CPCA_PROF("knn_to_half", st);
    to_half_kernel<<<unsigned(std::min<int64_t>(ceil_div(int64_t(N) * 32, 256), int64_t(num_sms()) * 16)), 256, 0,
                     st>>>(P, N, d, ld, w.hsc, w.H, ldh);
    CPCA_LAUNCHED();
    CPCA_TRY(knn_candidates_tc(w.H, N, d, ldh, w.hsc, M, S, w.nrm, w.cand_i, w.cand_d, w.err, &done, st));
  }
  if (!done) {
    const size_t smem = sizeof(float) * (BD * BQ + BD * BB + BQ * (BB + 1)) + size_t(BQ) * M * 8;
    dim3 grid(ceil_div(N, BQ), S);
    if (M == 32) {
      CPCA_CUDA(cudaFuncSetAttribute(knn_candidates_kernel<32>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      CPCA_PROF("knn_candidates_simt", st);
      knn_candidates_kernel<32><<<grid, KNN_THREADS, smem, st>>>(P, N, d, ld, w.nrm, S, w.cand_i, w.cand_d);
    } else {
      CPCA_CUDA(cudaFuncSetAttribute(knn_candidates_kernel<64>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      CPCA_PROF("knn_candidates_simt", st);
      knn_candidates_kernel<64><<<grid, KNN_THREADS, smem, st>>>(P, N, d, ld, w.nrm, S, w.cand_i, w.cand_d);
    }
    CPCA_LAUNCHED();
  }
  // FP32 expansion error model for the certificate: about 4 sqrt(d) + 16
  // roundings of size 2^-24 relative to |a|^2 + |b|^2 (the tensor-core pass
  // has its own, larger, bound: knn_tc_err_rel plus the absolute terms of
  // the half copy in hsc[2], hsc[3]).
  const float err_rel = done ? knn_tc_err_rel(d) : float((4.0 * sqrt(double(d)) + 16.0) * 0x1.0p-24);
  const float* err_abs = done ? w.hsc + 2 : nullptr;
  *err_rel_used = err_rel;
  const size_t rsm = size_t(RECHECK_WARPS) * S * M * 20;
  CPCA_CUDA(cudaFuncSetAttribute(knn_recheck_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(rsm)));
  CPCA_PROF("knn_recheck", st);
  knn_recheck_kernel<<<ceil_div(N, RECHECK_WARPS), RECHECK_WARPS * 32, rsm, st>>>(
      P, N, d, ld, vec4, K, M, S, w.cand_i, w.cand_d, w.nrm, w.nmax, err_rel, err_abs, out_i, out_d, w.redo,
      w.n_redo);
  CPCA_LAUNCHED();
  // queries without a certificate: how many, then, within the budget,
  // brute force in batches of kBfBatch over the whole grid. Beyond the
  // budget every such query keeps the exact K nearest of its S M
  // tensor-core candidates (re-scored in FP32, settled in FP64) and is
  // counted as uncertified.
  int nredo = 0;
  CPCA_CUDA(cudaMemcpyAsync(&nredo, w.n_redo, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  *n_bruteforce = 0;
  *n_uncertified = 0;
  if (nredo > knn_bruteforce_cap(N, d)) {
    *n_uncertified = nredo;
    return CPCA_OK;
  }
  *n_bruteforce = nredo;
  for (int r0 = 0; r0 < nredo; r0 += kBfBatch) {
    const int nq = std::min(kBfBatch, nredo - r0);
    // points per work item: enough items for about 32 warps per SM
    const int64_t want = int64_t(num_sms()) * 32;
    const int chunk = int(std::min<int64_t>(
        kBfChunkMax, std::max<int64_t>(kBfChunkMin, (ceil_div(int64_t(N) * nq, want) + 31) / 32 * 32)));
    const int64_t items = int64_t(nq) * ((N + chunk - 1) / chunk);
    const unsigned grid = unsigned(std::min<int64_t>((items + RECHECK_WARPS - 1) / RECHECK_WARPS, num_sms() * 16));
    CPCA_PROF("knn_bruteforce", st);
    knn_bf_score_kernel<<<grid, RECHECK_WARPS * 32, 0, st>>>(P, N, d, ld, vec4, w.redo, r0, nq, chunk, w.bf_d,
                                                              w.bf_i);
    CPCA_LAUNCHED();
    knn_bf_merge_kernel<<<ceil_div(nq, RECHECK_WARPS), RECHECK_WARPS * 32, 0, st>>>(
        P, N, d, ld, vec4, K, w.redo, r0, nq, chunk, w.bf_d, w.bf_i, out_i, out_d);
    CPCA_LAUNCHED();
  }
  return CPCA_OK;
}

// Graph + Laplacian from kNN lists.
cpca_status graph_from_knn(const int32_t* kidx, const float* kd2, int N, int K, int lap_type,
                           double sigma2, const KnnWs& w, int64_t* rowptr, int32_t* col,
                           float* val, float* weight, int64_t nnz_cap, cudaStream_t st) {
  const int64_t m = int64_t(N) * K;
  sum_partials_kernel<<<RED_BLOCKS, 256, 0, st>>>(kd2, m, w.part);
  CPCA_LAUNCHED();
  sigma2_finish_kernel<<<1, 32, 0, st>>>(w.part, RED_BLOCKS, m, sigma2, w.sigma2);
  CPCA_LAUNCHED();
  CPCA_CUDA(cudaMemsetAsync(w.indeg, 0, sizeof(int32_t) * N, st));
  CPCA_CUDA(cudaMemsetAsync(w.cursor, 0, sizeof(int32_t) * N, st));
  const unsigned eb = std::min<unsigned>(ceil_div(m, 256), num_sms() * 8);
  indeg_kernel<<<eb, 256, 0, st>>>(kidx, N, K, w.indeg);
  CPCA_LAUNCHED();
  scan_kernel<<<1, 1024, 0, st>>>(w.indeg, K, N, w.off);
  CPCA_LAUNCHED();
  fill_edges_kernel<<<eb, 256, 0, st>>>(kidx, kd2, N, K, w.off, w.cursor, w.e_nbr, w.e_d2);
  CPCA_LAUNCHED();
  CPCA_PROF("graph_dedupe", st);
  CPCA_CUDA(cudaMemsetAsync(w.n_long, 0, sizeof(int32_t), st));
  dedupe_kernel<<<unsigned(std::min<int64_t>(ceil_div(int64_t(N) * 32, 256), int64_t(num_sms()) * 16)), 256, 0, st>>>(
      N, w.off, w.e_nbr, w.e_d2, w.uniq, w.longq, w.n_long);
  CPCA_LAUNCHED();
  {
    const size_t lsm = size_t(kDedupeBlockMax) * (sizeof(unsigned long long) + sizeof(float));
    static PerDeviceOnce attr;
    CPCA_CUDA(once_per_device(attr, [&] {
      return cudaFuncSetAttribute(dedupe_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lsm));
    }));
    dedupe_long_kernel<<<num_sms(), 1024, lsm, st>>>(w.off, w.e_nbr, w.e_d2, w.uniq, w.longq, w.n_long);
    CPCA_LAUNCHED();
  }
  scan_kernel<<<1, 1024, 0, st>>>(w.uniq, 1, N, rowptr);
  CPCA_LAUNCHED();
  degree_kernel<<<ceil_div(N, 128), 128, 0, st>>>(N, w.off, w.uniq, w.e_d2, w.sigma2, w.deg);
  CPCA_LAUNCHED();
  CPCA_PROF("graph_assemble", st);
  assemble_kernel<<<ceil_div(N, 128), 128, 0, st>>>(N, lap_type, w.off, w.uniq, w.e_nbr, w.e_d2,
                                                    w.sigma2, w.deg, rowptr, nnz_cap, col, val, weight);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

}  // namespace cpca

using namespace cpca;

static thread_local int g_knn_last_redo = 0;
static thread_local int g_knn_last_unc = 0;
static thread_local double g_knn_last_err_rel = 0.0;

extern "C" int32_t cpca_knn_last_bruteforce(void) { return g_knn_last_redo; }
extern "C" int32_t cpca_knn_last_uncertified(void) { return g_knn_last_unc; }
extern "C" double cpca_knn_last_err_rel(void) { return g_knn_last_err_rel; }

extern "C" size_t cpca_knn_graph_workspace_size(int32_t npts, int32_t dim, int32_t K,
                                                int32_t transposed) {
  if (npts <= 0 || dim <= 0 || K <= 0) return 0;
  return knn_layout(nullptr, npts, dim, K, transposed).bytes;
}

extern "C" cpca_status cpca_knn_graph(const float* pts, int32_t npts, int32_t dim, int64_t ld,
                                      int32_t transposed, int32_t K, int32_t lap_type,
                                      double sigma2, int64_t* rowptr, int32_t* col, float* val,
                                      float* weight, int64_t nnz_cap, int32_t* knn_idx,
                                      float* knn_d2, int64_t* nnz_out, double* sigma2_out,
                                      void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_knn_graph");
  CPCA_CHECK_ARG(pts && rowptr && col && val, "cpca_knn_graph: null pointer");
  CPCA_CHECK_ARG(npts >= 2 && dim >= 1, "cpca_knn_graph: need npts >= 2, dim >= 1");
  CPCA_CHECK_ARG(K >= 1 && K <= 32 && K < npts, "cpca_knn_graph: need 1 <= K <= 32, K < npts");
  CPCA_CHECK_ARG(transposed == 0 || transposed == 1, "cpca_knn_graph: transposed must be 0/1");
  CPCA_CHECK_ARG(ld >= (transposed ? npts : dim), "cpca_knn_graph: leading dimension too small");
  CPCA_CHECK_ARG(lap_type == CPCA_LAP_NORMALIZED || lap_type == CPCA_LAP_COMBINATORIAL,
                 "cpca_knn_graph: bad lap_type");
  CPCA_CHECK_ARG(nnz_cap >= int64_t(npts) * (2 * K + 1), "cpca_knn_graph: nnz_cap < npts*(2K+1)");
  const KnnWs w = knn_layout(ws, npts, dim, K, transposed);
  if (ws_bytes < w.bytes || !ws) {
    set_error("cpca_knn_graph: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float* P = pts;
  int64_t pld = ld;
  if (transposed) {
    // Point-major copy of the columns (rows of length dim, ld = dim).
    // rows padded with zeros to a multiple of 4 floats (16-byte row stride)
    const int dpad = (dim + 3) & ~3;
    if (dpad != dim) CPCA_CUDA(cudaMemsetAsync(w.Pt, 0, sizeof(float) * size_t(npts) * dpad, st));
    dim3 blk(32, 8), grd(ceil_div(npts, 32), ceil_div(dim, 32));
    CPCA_PROF("knn_transpose", st);
    transpose_kernel<<<grd, blk, 0, st>>>(pts, dim, npts, ld, w.Pt, dpad);
    CPCA_LAUNCHED();
    P = w.Pt;
    pld = dpad;
  }
  int32_t* oi = knn_idx ? knn_idx : w.kidx;
  float* od = knn_d2 ? knn_d2 : w.kd2;
  int nbf = 0, nunc = 0;
  float erel = 0.f;
  CPCA_TRY(knn_lists(P, npts, dim, pld, K, w, oi, od, &nbf, &nunc, &erel, st));
  g_knn_last_redo = nbf;
  g_knn_last_unc = nunc;
  g_knn_last_err_rel = erel;
  CPCA_TRY(graph_from_knn(oi, od, npts, K, lap_type, sigma2, w, rowptr, col, val, weight, nnz_cap, st));
  int64_t nnz = 0;
  double s2 = 0;
  CPCA_CUDA(cudaMemcpyAsync(&nnz, rowptr + npts, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(&s2, w.sigma2, sizeof(double), cudaMemcpyDeviceToHost, st));
  int terr = 0;
  CPCA_CUDA(cudaMemcpyAsync(&terr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (terr) {
    set_error("cpca_knn_graph: tensor-core pass timed out waiting on an mbarrier");
    return CPCA_ERR_TIMEOUT;
  }
  if (nnz_out) *nnz_out = nnz;
  if (sigma2_out) *sigma2_out = s2;
  if (nnz > nnz_cap) {
    set_error("cpca_knn_graph: nnz %lld exceeds nnz_cap %lld", (long long)nnz, (long long)nnz_cap);
    return CPCA_ERR_CAPACITY;
  }
  return CPCA_OK;
}
