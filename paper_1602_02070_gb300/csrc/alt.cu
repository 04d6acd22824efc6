// alt.cu - the alternate decoder (Sec. V-B, Eq. alternatedecoder): the full
// p x n matrix X minimising
//   |M_r X M_c - X~|_F^2 + gc tr(X L_c X^T) + gr tr(X^T L_r X),
// i.e. the solution of the normal equations
//   A(X) = D_r X D_c + gc X L_c + gr L_r X = M_r^T X~ M_c^T = B,
// D_r, D_c the 0/1 diagonals of the sampled rows and columns, solved by
// Jacobi-preconditioned conjugate gradients (the paper names CG for it).
//
// One persistent cooperative launch runs the whole solve over 32 x 32 tiles
// of X (column-block-major order), two grid barriers per iteration. With
// z = M^{-1} r and p_new = z + beta p, the operator is applied to z, not to
// p: A p_new = A z + beta A p_old, so only z has to be published in both
// layouts (row-major for the L_r gathers, column-major for the L_c ones,
// as in the FISTA kernel), and p and q = A p stay in their own tiles.
//   phase A (tile): w = A z (gathers), q = w + beta q, p = z + beta p,
//                   partial p^T q;                          grid barrier
//   phase B (tile): alpha = r^T z / p^T q, x += alpha p, r -= alpha q,
//                   z = r / diag(A), z published, partials r^T z, r^T r;
//                                                           grid barrier
// Dot products are FP64 partial sums per block, added up in block order by
// every block (the same bits everywhere, so every block takes the same
// convergence decision). Stop: |r|_2 <= tol |B|_2.
#include <algorithm>
#include <cmath>

#include "fista_internal.cuh"

namespace cpca {
namespace {

constexpr int kAltMaxBlocks = 2048;

struct AltArgs {
  const float* Xt;
  int64_t ldxt;
  const int* srow;  // position of row i in Omega_r, or -1
  const int* scol;  // position of column j in Omega_c, or -1
  const float* dr;  // diagonal of L_r
  const float* dc;  // diagonal of L_c
  CsrView Lr, Lc;
  int p, n, nti, ntiles;
  int64_t ldz, ldzt;  // padded row lengths (multiples of 4)
  float gr, gc;
  float *x, *r, *pv, *q, *z, *zt;
  double* part;  // [3][kAltMaxBlocks]: r^T z, p^T q, r^T r (B^T B in the setup)
  double* out;   // [4]: final r^T r, B^T B, iterations, converged
  double tol2;
  int max_iter;
  float* X;
  int64_t ldx;
  int xvec;
  GridBar bar;
};

struct AltSmem {
  TileNbr nb;
  float ac[TB][TB + 1];  // (z L_c) of the tile, [row][col]
  float tl[TB][TB + 1];  // tile of z for the transposed store
  double red[8];
  double bc[3];
};

__device__ __forceinline__ float4 ld4v(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4v(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& c4(float4& v, int t) { return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w; }

// Sum of part[0..nb) in block order by warp 0, broadcast through shared memory.
__device__ __forceinline__ double all_sum(const double* part, int nb, double* slot) {
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) t += __ldcg(part + b);
    t = warp_sum(t);
    if (threadIdx.x == 0) *slot = t;
  }
  __syncthreads();
  return *slot;
}

__device__ __forceinline__ void tile_at(const AltArgs& a, int t, int& i0, int& j0, int& ni, int& nj) {
  i0 = (t % a.nti) * TB;
  j0 = (t / a.nti) * TB;
  ni = min(TB, a.p - i0);
  nj = min(TB, a.n - j0);
}

// transposed store of the tile's z through shared memory
__device__ __forceinline__ void publish_zt(AltSmem& sm, const AltArgs& a, float4 z4, int rl, int cq, int i0,
                                           int j0, int ni, int nj) {
  sm.tl[rl][cq] = z4.x;
  sm.tl[rl][cq + 1] = z4.y;
  sm.tl[rl][cq + 2] = z4.z;
  sm.tl[rl][cq + 3] = z4.w;
  __syncthreads();
  if (rl < nj && cq < ni)
    st4v(a.zt + int64_t(j0 + rl) * a.ldzt + i0 + cq,
         make_float4(sm.tl[cq][rl], sm.tl[cq + 1][rl], sm.tl[cq + 2][rl], sm.tl[cq + 3][rl]));
  __syncthreads();
}

__global__ void __launch_bounds__(256, 4) alt_cg_kernel(const __grid_constant__ AltArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  AltSmem& sm = *reinterpret_cast<AltSmem*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = warp * 4 + (lane >> 3), cq = 4 * (lane & 7);
  const int nb = gridDim.x;
  double* Prz = a.part;
  double* Ppq = a.part + kAltMaxBlocks;
  double* Prr = a.part + 2 * kAltMaxBlocks;
  // diagonal of A at 4 entries of row i: mask + gc L_c(j, j) + gr L_r(i, i)
  auto diag4 = [&](int i, int64_t jj, int nv, float4& m4) {
    float4 d4 = make_float4(1.f, 1.f, 1.f, 1.f);
    const bool rs = a.srow[i] >= 0;
    const float gri = a.gr * a.dr[i];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < nv) {
        const float m = (rs && a.scol[jj + t] >= 0) ? 1.f : 0.f;
        c4(m4, t) = m;
        c4(d4, t) = m + a.gc * a.dc[jj + t] + gri;
      }
    return d4;
  };

  // setup: x = 0, r = B, z = M^{-1} r, p = q = 0; partials r^T z and B^T B
  {
    double rz = 0.0, bb = 0.0;
    for (int t = blockIdx.x; t < a.ntiles; t += nb) {
      int i0, j0, ni, nj;
      tile_at(a, t, i0, j0, ni, nj);
      float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rl < ni && cq < nj) {
        const int i = i0 + rl;
        const int64_t jj = j0 + cq, l = int64_t(i) * a.ldz + jj;
        const int nv = nj - cq;
        float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f), b4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 d4 = diag4(i, jj, nv, m4);
        const int si = a.srow[i];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nv && c4(m4, u) != 0.f) c4(b4, u) = a.Xt[int64_t(si) * a.ldxt + a.scol[jj + u]];
        float4 dd = d4;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float d = c4(dd, u);
          c4(z4, u) = u < nv ? (d > 0.f ? c4(b4, u) / d : c4(b4, u)) : 0.f;
          rz += double(c4(b4, u)) * double(c4(z4, u));
          bb += double(c4(b4, u)) * double(c4(b4, u));
        }
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        st4v(a.x + l, zero);
        st4v(a.pv + l, zero);
        st4v(a.q + l, zero);
        st4v(a.r + l, b4);
        st4v(a.z + l, z4);
      }
      publish_zt(sm, a, z4, rl, cq, i0, j0, ni, nj);
    }
    rz = block_sum(rz, sm.red);
    bb = block_sum(bb, sm.red);
    if (threadIdx.x == 0) {
      Prz[blockIdx.x] = rz;
      Prr[blockIdx.x] = bb;
    }
  }
  if (!grid_sync(a.bar)) return;
  const double bb = all_sum(Prr, nb, &sm.bc[2]);
  double rz = all_sum(Prz, nb, &sm.bc[0]);
  double rz_prev = 1.0, rr = bb;
  int k = 0;
  bool conv = bb <= a.tol2 * bb || bb == 0.0;
  for (; k < a.max_iter && !conv; ++k) {
    const float beta = k == 0 ? 0.f : float(rz / rz_prev);
    // phase A: q = A z + beta q, p = z + beta p
    double pq = 0.0;
    for (int t = blockIdx.x; t < a.ntiles; t += nb) {
      int i0, j0, ni, nj;
      tile_at(a, t, i0, j0, ni, nj);
      stage_nbr(sm.nb, a.Lr, a.Lc, int(a.ldzt), int(a.ldz), i0, j0, ni, nj);
      {
        const float4 o = nbr_sum_v4<int64_t, 8>(sm.nb.coff[rl], sm.nb.cval[rl], sm.nb.cdeg[rl], sm.nb.cf0[rl],
                                                rl < nj && cq < ni, a.zt, i0 + cq, a.Lc, a.ldzt);
        sm.ac[cq][rl] = o.x;
        sm.ac[cq + 1][rl] = o.y;
        sm.ac[cq + 2][rl] = o.z;
        sm.ac[cq + 3][rl] = o.w;
      }
      const bool own = rl < ni && cq < nj;
      const float4 ar = nbr_sum_v4<int64_t, 8>(sm.nb.roff[rl], sm.nb.rval[rl], sm.nb.rdeg[rl], sm.nb.rf0[rl], own,
                                               a.z, j0 + cq, a.Lr, a.ldz);
      __syncthreads();
      if (own) {
        const int i = i0 + rl;
        const int64_t jj = j0 + cq, l = int64_t(i) * a.ldz + jj;
        const int nv = nj - cq;
        float4 z4 = __ldcg(reinterpret_cast<const float4*>(a.z + l));
        float4 q4 = ld4v(a.q + l), p4 = ld4v(a.pv + l);
        const bool rs = a.srow[i] >= 0;
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f), pn = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 arr = ar;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nv) {
            const float m = (rs && a.scol[jj + u] >= 0) ? c4(z4, u) : 0.f;
            const float w = fmaf(a.gr, c4(arr, u), fmaf(a.gc, sm.ac[rl][cq + u], m));
            c4(qn, u) = fmaf(beta, c4(q4, u), w);
            c4(pn, u) = fmaf(beta, c4(p4, u), c4(z4, u));
            pq += double(c4(pn, u)) * double(c4(qn, u));
          }
        st4v(a.q + l, qn);
        st4v(a.pv + l, pn);
      }
      __syncthreads();  // the lists and sm.ac are reused by the next tile
    }
    pq = block_sum(pq, sm.red);
    if (threadIdx.x == 0) Ppq[blockIdx.x] = pq;
    if (!grid_sync(a.bar)) return;
    const double pqs = all_sum(Ppq, nb, &sm.bc[1]);
    const float alpha = pqs > 0.0 ? float(rz / pqs) : 0.f;
    // phase B: x += alpha p, r -= alpha q, z = M^{-1} r (published)
    double rzn = 0.0, rrn = 0.0;
    for (int t = blockIdx.x; t < a.ntiles; t += nb) {
      int i0, j0, ni, nj;
      tile_at(a, t, i0, j0, ni, nj);
      float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rl < ni && cq < nj) {
        const int i = i0 + rl;
        const int64_t jj = j0 + cq, l = int64_t(i) * a.ldz + jj;
        const int nv = nj - cq;
        float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 d4 = diag4(i, jj, nv, m4);
        float4 x4 = ld4v(a.x + l), r4 = ld4v(a.r + l);
        const float4 p4 = ld4v(a.pv + l), q4 = ld4v(a.q + l);
        float4 pp = p4, qq = q4, dd = d4;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nv) {
            c4(x4, u) = fmaf(alpha, c4(pp, u), c4(x4, u));
            const float rv = fmaf(-alpha, c4(qq, u), c4(r4, u));
            c4(r4, u) = rv;
            const float d = c4(dd, u);
            const float zv = d > 0.f ? rv / d : rv;
            c4(z4, u) = zv;
            rzn += double(rv) * double(zv);
            rrn += double(rv) * double(rv);
          }
        st4v(a.x + l, x4);
        st4v(a.r + l, r4);
        st4v(a.z + l, z4);
      }
      publish_zt(sm, a, z4, rl, cq, i0, j0, ni, nj);
    }
    rzn = block_sum(rzn, sm.red);
    rrn = block_sum(rrn, sm.red);
    if (threadIdx.x == 0) {
      Prz[blockIdx.x] = rzn;
      Prr[blockIdx.x] = rrn;
    }
    if (!grid_sync(a.bar)) return;
    rz_prev = rz;
    rz = all_sum(Prz, nb, &sm.bc[0]);
    rr = all_sum(Prr, nb, &sm.bc[2]);
    conv = rr <= a.tol2 * bb;
  }
  // X = x
  for (int t = blockIdx.x; t < a.ntiles; t += nb) {
    int i0, j0, ni, nj;
    tile_at(a, t, i0, j0, ni, nj);
    if (rl < ni && cq < nj) {
      const int i = i0 + rl;
      const int64_t jj = j0 + cq;
      const int nv = nj - cq;
      float4 x4 = ld4v(a.x + int64_t(i) * a.ldz + jj);
      float* dst = a.X + int64_t(i) * a.ldx + jj;
      if (a.xvec) {
        st4v(dst, x4);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nv) dst[u] = c4(x4, u);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = rr;
    a.out[1] = bb;
    a.out[2] = double(k);
    a.out[3] = conv ? 1.0 : 0.0;
  }
}

// srow[omega[t]] = t (sampled positions); out-of-range or repeated indices
// set *bad and are skipped
__global__ void alt_scatter_kernel(const int* __restrict__ omega, int m, int N, int* __restrict__ pos,
                                   int* __restrict__ bad) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const int v = omega[t];
    if (v < 0 || v >= N) {
      atomicExch(bad, 1);
      continue;
    }
    if (atomicCAS(pos + v, -1, t) != -1) atomicExch(bad, 1);
  }
}

// d[i] = L(i, i) (0 where the row stores no diagonal entry)
__global__ void alt_diag_kernel(CsrView L, float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e)
      if (L.col[e] == i) v = L.val[e];
    d[i] = v;
  }
}

struct AltWs {
  float *x, *r, *pv, *q, *z, *zt, *dr, *dc;
  int *srow, *scol;
  double *part, *out;
  unsigned int* bar;
  int* err;
  int* bad;
  size_t bytes;
};

AltWs alt_layout(void* ws, int p, int n) {
  Carve c(ws);
  AltWs w{};
  const size_t mn = size_t(p) * ((n + 3) / 4 * 4), mnt = size_t(n) * ((p + 3) / 4 * 4);
  w.x = c.take<float>(mn);
  w.r = c.take<float>(mn);
  w.pv = c.take<float>(mn);
  w.q = c.take<float>(mn);
  w.z = c.take<float>(mn);
  w.zt = c.take<float>(mnt);
  w.dr = c.take<float>(p);
  w.dc = c.take<float>(n);
  w.srow = c.take<int>(p);
  w.scol = c.take<int>(n);
  w.part = c.take<double>(3 * kAltMaxBlocks);
  w.out = c.take<double>(4);
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.bad = c.take<int>(1);
  w.bytes = c.bytes();
  return w;
}

}  // namespace
}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_alternate_decode_workspace_size(int32_t p, int32_t n) {
  if (p <= 0 || n <= 0) return 0;
  return alt_layout(nullptr, p, n).bytes;
}

extern "C" cpca_status cpca_alternate_decode(const float* Xt, int32_t rr, int32_t rc, int64_t ldxt,
                                             const int32_t* omega_r, const int32_t* omega_c, int32_t p,
                                             int32_t n, const cpca_csr* Lr, const cpca_csr* Lc,
                                             const cpca_alt_params* prm, float* X, int64_t ldx,
                                             cpca_alt_info* info, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_alternate_decode");
  CPCA_CHECK_ARG(Xt && omega_r && omega_c && X && prm, "cpca_alternate_decode: null pointer");
  CPCA_CHECK_ARG(p > 0 && n > 0 && rr > 0 && rc > 0 && rr <= p && rc <= n,
                 "cpca_alternate_decode: bad sizes (p %d, n %d, rr %d, rc %d)", p, n, rr, rc);
  CPCA_CHECK_ARG(ldxt >= rc && ldx >= n, "cpca_alternate_decode: leading dimension too small");
  CPCA_CHECK_ARG(prm->gamma_r >= 0 && prm->gamma_c >= 0 && prm->tol >= 0 && prm->max_iter >= 0,
                 "cpca_alternate_decode: bad parameters");
  CPCA_TRY(check_csr(Lr, p, "cpca_alternate_decode(Lr)"));
  CPCA_TRY(check_csr(Lc, n, "cpca_alternate_decode(Lc)"));
  const AltWs w = alt_layout(ws, p, n);
  if (!ws || ws_bytes < w.bytes) {
    set_error("cpca_alternate_decode: workspace %zu bytes < required %zu", ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const CsrView lr{Lr->n, Lr->rowptr, Lr->col, Lr->val}, lc{Lc->n, Lc->rowptr, Lc->col, Lc->val};
  CPCA_CUDA(cudaMemsetAsync(w.srow, 0xff, sizeof(int) * p, st));
  CPCA_CUDA(cudaMemsetAsync(w.scol, 0xff, sizeof(int) * n, st));
  CPCA_CUDA(cudaMemsetAsync(w.bad, 0, sizeof(int), st));
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  CPCA_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  CPCA_PROF("alt_setup", st);
  alt_scatter_kernel<<<std::max(1u, std::min(ceil_div(rr, 256), 64u)), 256, 0, st>>>(omega_r, rr, p, w.srow, w.bad);
  CPCA_LAUNCHED();
  alt_scatter_kernel<<<std::max(1u, std::min(ceil_div(rc, 256), 64u)), 256, 0, st>>>(omega_c, rc, n, w.scol, w.bad);
  CPCA_LAUNCHED();
  alt_diag_kernel<<<std::min(ceil_div(p, 256), 1024u), 256, 0, st>>>(lr, w.dr);
  CPCA_LAUNCHED();
  alt_diag_kernel<<<std::min(ceil_div(n, 256), 1024u), 256, 0, st>>>(lc, w.dc);
  CPCA_LAUNCHED();
  int bad = 0;
  CPCA_CUDA(cudaMemcpyAsync(&bad, w.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (bad) {
    set_error("cpca_alternate_decode: omega indices out of range or repeated");
    return CPCA_ERR_INVALID_ARG;
  }
  AltArgs a{};
  a.Xt = Xt;
  a.ldxt = ldxt;
  a.srow = w.srow;
  a.scol = w.scol;
  a.dr = w.dr;
  a.dc = w.dc;
  a.Lr = lr;
  a.Lc = lc;
  a.p = p;
  a.n = n;
  a.nti = int(ceil_div(p, TB));
  a.ntiles = int(int64_t(a.nti) * ceil_div(n, TB));
  a.ldz = (n + 3) / 4 * 4;
  a.ldzt = (p + 3) / 4 * 4;
  a.gr = float(prm->gamma_r);
  a.gc = float(prm->gamma_c);
  a.x = w.x;
  a.r = w.r;
  a.pv = w.pv;
  a.q = w.q;
  a.z = w.z;
  a.zt = w.zt;
  a.part = w.part;
  a.out = w.out;
  a.tol2 = prm->tol * prm->tol;
  a.max_iter = prm->max_iter;
  a.X = X;
  a.ldx = ldx;
  a.xvec = ldx % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
  a.bar = grid_bar(w.bar, w.err);
  const size_t smem = sizeof(AltSmem);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    return cudaFuncSetAttribute((const void*)alt_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  }));
  int grid = coop_blocks((const void*)alt_cg_kernel, 256, smem, std::min(a.ntiles, kAltMaxBlocks));
  if (prm->blocks > 0) grid = std::min(grid, int(prm->blocks));
  void* args[] = {&a};
  CPCA_PROF("alt_cg", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)alt_cg_kernel, dim3(grid), dim3(256), args, smem, st));
  CPCA_LAUNCHED();
  double out[4] = {0, 0, 0, 0};
  int err = 0;
  CPCA_CUDA(cudaMemcpyAsync(out, w.out, sizeof(out), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("cpca_alternate_decode: grid barrier timed out");
    return CPCA_ERR_TIMEOUT;
  }
  if (info) {
    info->iters = int32_t(out[2]);
    info->rel_res = out[1] > 0 ? std::sqrt(out[0] / out[1]) : 0.0;
    info->converged = out[3] != 0.0;
  }
  if (out[3] == 0.0) {
    set_error("cpca_alternate_decode: no convergence in %d iterations", prm->max_iter);
    return CPCA_ERR_NOT_CONVERGED;
  }
  return CPCA_OK;
}
