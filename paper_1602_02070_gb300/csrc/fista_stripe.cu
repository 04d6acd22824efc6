// fista_stripe.cu - FISTA for FRPCAG (Sec. IV-B, Algorithm 1) on single
// problems too large for the resident launch, one launch per iteration.
//
// Layout. The columns are taken in a processing order (the column graph's
// locality order from order.cu for large problems, else the identity) and
// cut into stripes of W = 16 (or 8) columns. Y~, S, the previous iterate
// and Z_j are held stripe-major for the solve: stripe s is one contiguous
// block of rr x W floats, row i of it at (s rr + i) W. Z_j^T is kept as well
// (column-major, rows padded to ldzt), for the column graph's gathers. The
// caller's matrices are converted in at the start and S out at the end.
//
// One block per SM (1024 threads) takes stripes in turn (the next untaken
// one when it finishes its last). For each it
// brings the stripe of Z_j into shared memory with one bulk copy (the block
// is contiguous) and stages the stripe columns' neighbour lists (as Z^T row
// offsets), then in chunks of 1024 rows:
//   (Z Lc)(i, c) = sum_l Lc[c, l] Z^T(l, i): work items (column, row block)
//       that the warps take in turn - 256 rows (a lane per 8 rows, two
//       16-byte loads per neighbour) for a column with a short list, 64 rows
//       (a lane per 2 rows, 8-byte loads) for one with a long list, so that
//       the hub columns of a kNN graph spread over the warps; the
//       neighbours' Z^T rows are read through L1
//       (neighbouring columns of the stripe share them); overlaps the
//       stripe's copy on the first chunk;
//   (Lr Z)(i, c) = sum_k Lr[i, k] Z(k, c): W/4 lanes per row, each a quad
//       of 4 columns, entirely from the stripe in shared memory (a row
//       graph links arbitrary rows and the stripe holds all of them): a
//       lane group reads one contiguous stripe row per entry, and the
//       groups of a warp spread over the banks;
//   S_j = prox(Z_j - lambda 2 (g_c Z Lc + g_r Lr Z)),
//   Z_{j+1} = S_j + mu_j (S_j - S_{j-1}),
// written stripe-major (S_j, Z_{j+1}) and column-major (Z_{j+1}^T). Both
// graph sums run in CSR order with one FMA per entry from zero, exactly as
// the cooperative kernel's: the iterates are bit for bit those of
// fista_batch_kernel (the processing order moves data, not arithmetic).
// Launch boundaries order the iterations, so there is no grid barrier; with
// eps > 0 every launch first reads the previous iteration's statistics and
// all its blocks leave once the stopping test holds.
//
// Bytes per entry and iteration: read Y~, S_{j-1}, Z_j (stripe) and Z_j^T
// (gathers, once from DRAM when the rows in flight stay in L2), write S_j,
// Z_{j+1}, Z_{j+1}^T: 28 B, against the method's 16 B (Y~, S_{j-1},
// S_{j-2} in, S_j out); plus the CSR bytes.
#include "fista_internal.cuh"
#include "tma.cuh"

namespace cpca {
namespace {

// Launch shape per stripe width: W = 16 - one block of 1024 threads per SM,
// chunks of 1024 rows; W = 8 - two blocks of 512 threads per SM (each with
// its own stripe, so that one block's gathers overlap the other's shared-
// memory work), chunks of 512 rows.
template <int W>
struct Shape {
  static constexpr int ST = W == 16 ? 1024 : 512;  // threads per block
  static constexpr int RC = ST;                    // rows per chunk
  static constexpr int BLOCKS = W == 16 ? 1 : 2;   // blocks per SM
};
constexpr int kPool = 2048;     // staged neighbour entries per stripe
constexpr int kHubDeg = 48;     // columns with longer lists take 32-row items
constexpr uint32_t kBulk = 32768;  // bytes per bulk copy of a stripe

struct StripeArgs {
  const float* Zin;   // Z_j, stripe-major
  const float* ZTin;  // Z_j^T, [rc][ldzt], processing order
  float* Zout;        // Z_{j+1}, stripe-major
  float* ZTout;       // Z_{j+1}^T
  const float* Yb;    // Y~, stripe-major
  float* Sb;          // S_{j-1} in, S_j out, stripe-major
  float* Pb;          // S_{J-1} on the last iteration (stripe-major), or null
  CsrView Lr, Lc;
  const int32_t* perm;  // processing position -> column of Lc (null: identity)
  const int32_t* inv;   // column of Lc -> processing position
  const double* lam;
  double* stats;  // ring [4][2]
  int* done;      // [stopped, iterations]
  int* err;       // mbarrier timeout flag
  unsigned int* ctr;  // stripe counters, a ring of three (launch j takes j % 3)
  int64_t ldzt;
  float two_gr, two_gc, mu;
  int rr, rc, nstripes;
  int nfull, nunits;  // work units: whole stripes [0, nfull), then halves of the rest
  int j, J;
  double eps;
  int want_stats;
};

template <int W>
struct StripeSmem {
  float ac[W][Shape<W>::RC];  // (Z Lc) of the chunk, [column][row]
  int2 pool[kPool];       // the stripe's neighbour lists, column after column in CSR
                          // order: (element offset of the Z^T row, weight bits)
  int64_t cf0[W];         // first CSR entry of each stripe column
  int cdeg[W], cbeg[W];   // its degree and its first pool slot
  int hubc[W], normc[W];  // columns taken in 32-row items (long lists) / 128-row items
  int nhub, nnorm, next;  // their counts; the next column-product item
  int next_stripe;
  uint64_t mbar;
  double red[2][Shape<W>::ST / 32];
  int abort;
};

template <int W>
__host__ __device__ constexpr size_t smem_head() {
  return (sizeof(StripeSmem<W>) + 127) & ~size_t(127);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void fma4(float4& acc, float w, const float4& v) {
  acc.x = fmaf(w, v.x, acc.x);
  acc.y = fmaf(w, v.y, acc.y);
  acc.z = fmaf(w, v.z, acc.z);
  acc.w = fmaf(w, v.w, acc.w);
}

// One prox + momentum entry of Algorithm 1 (the cooperative kernel's
// expression order).
__device__ __forceinline__ void prox_entry(float ar, float ac, float z, float y, float sp, float lam, float two_gr,
                                           float two_gc, float mu, float& sv, float& zn) {
  const float gr = fmaf(two_gr, ar, two_gc * ac);
  const float v = fmaf(-lam, gr, z);
  const float dl = v - y;
  sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
  zn = fmaf(mu, sv - sp, sv);
}

template <int W>
__global__ void __launch_bounds__(Shape<W>::ST, Shape<W>::BLOCKS)
    fista_stripe_kernel(const __grid_constant__ StripeArgs a) {
  constexpr int ST = Shape<W>::ST, RC = Shape<W>::RC;
  constexpr int NQ = W / 4;        // 16-byte quads per stripe row
  extern __shared__ __align__(128) unsigned char smraw[];
  StripeSmem<W>& sm = *reinterpret_cast<StripeSmem<W>*>(smraw);
  float* zs = reinterpret_cast<float*>(smraw + smem_head<W>());
  int32_t* rowp = reinterpret_cast<int32_t*>(zs + size_t(a.rr) * W);  // [rr + 1], from rowptr[0]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (__ldcg(a.done)) return;  // stopped at an earlier iteration
  if (a.eps > 0 && a.j > 1) {
    const double* ps = a.stats + 2 * ((a.j - 1) & 3);
    if (ps[0] < a.eps * ps[1]) {  // the same decision in every block
      if (blockIdx.x == 0 && tid == 0) {
        a.done[1] = a.j - 1;
        a.done[0] = 1;
      }
      return;
    }
  }
  // the statistics slot of iteration j + 1 (its last reader was iteration j - 2)
  if (blockIdx.x == 0 && tid < 2) a.stats[2 * ((a.j + 1) & 3) + tid] = 0.0;
  // the stripe counter of launch j + 1 (its last user was launch j - 2)
  if (blockIdx.x == 0 && tid == 0) a.ctr[(a.j + 1) % 3] = 0u;
  const float lam = float(*a.lam);
  const uint32_t stripe_bytes = uint32_t(a.rr) * W * 4;
  if (tid == 0) {
    sm.abort = 0;
    mbar_init(&sm.mbar, 1);
    mbar_fence_init();
  }
  const int64_t rbase = a.Lr.rowptr[0];
  for (int i = tid; i <= a.rr; i += ST) rowp[i] = int32_t(a.Lr.rowptr[i] - rbase);
  __syncthreads();
  // unit u: stripe u (u < nfull), else the half (u - nfull) % 2 of stripe
  // nfull + (u - nfull) / 2, rows [0, rh) or [rh, rr) (the last wave of
  // stripes in halves, so that blocks finish closer together)
  const int rh = ((a.rr + 1) / 2 + 3) / 4 * 4;
  auto unit_stripe = [&](int u) { return u < a.nfull ? u : a.nfull + (u - a.nfull) / 2; };
  auto issue = [&](int u) {  // one thread: the whole stripe of unit u into the buffer
    const char* src = reinterpret_cast<const char*>(a.Zin + int64_t(unit_stripe(u)) * a.rr * W);
    mbar_expect_tx(&sm.mbar, stripe_bytes);
    for (uint32_t o = 0; o < stripe_bytes; o += kBulk)
      bulk_load(reinterpret_cast<char*>(zs) + o, src + o, min(kBulk, stripe_bytes - o), &sm.mbar);
  };
  if (tid == 0 && int(blockIdx.x) < a.nunits) issue(blockIdx.x);
  double dz = 0.0, nz = 0.0;
  int k = 0;
  // the first unit of a block is its index; then blocks take the next
  // untaken unit as they finish (stripes with hub columns cost more)
  for (int u = blockIdx.x; u < a.nunits; ++k) {
    const int s = unit_stripe(u), c0 = s * W;
    const int rlo = u < a.nfull || ((u - a.nfull) & 1) == 0 ? 0 : rh;
    const int rhi = u < a.nfull || ((u - a.nfull) & 1) == 1 ? a.rr : rh;
    // neighbour lists of the stripe's columns, into the pool as far as it
    // holds them (the rest is read from the CSR as it is needed)
    if (tid < W) {
      const int jp = c0 + tid;
      const int jc = jp < a.rc ? (a.perm ? a.perm[jp] : jp) : 0;
      const int64_t f0 = jp < a.rc ? a.Lc.rowptr[jc] : 0;
      sm.cf0[tid] = f0;
      sm.cdeg[tid] = jp < a.rc ? int(a.Lc.rowptr[jc + 1] - f0) : 0;
    }
    __syncthreads();
    if (tid == 0) {
      int b = 0, nh = 0, nn = 0;
      for (int c = 0; c < W; ++c) {
        sm.cbeg[c] = b;
        b += sm.cdeg[c];
        if (sm.cdeg[c] > kHubDeg) sm.hubc[nh++] = c;
        else sm.normc[nn++] = c;
      }
      sm.nhub = nh;
      sm.nnorm = nn;
      sm.next = 0;
    }
    __syncthreads();
    {
      const int total = min(sm.cbeg[W - 1] + sm.cdeg[W - 1], kPool);
      for (int e = tid; e < total; e += ST) {
        int c = 0;
        while (c + 1 < W && sm.cbeg[c + 1] <= e) ++c;
        const int64_t f = sm.cf0[c] + (e - sm.cbeg[c]);
        const int l = __ldg(a.Lc.col + f);
        sm.pool[e] = make_int2(int32_t(a.inv ? a.inv[l] : l) * int32_t(a.ldzt), __float_as_int(__ldg(a.Lc.val + f)));
      }
    }
    __syncthreads();
    bool loaded = false;
    for (int r0 = rlo; r0 < rhi; r0 += RC) {
      const int nr = min(RC, rhi - r0);
      // ---- (Z Lc): items (column, row block) taken by the warps in turn: a
      // column with a short list in 256-row items (a lane per 8 rows, two
      // 16-byte loads per neighbour), one with a long list in 64-row items (a
      // lane per 2 rows, 8-byte loads), so that long lists spread over many
      // warps; every output still sums its column's list in CSR order.
      {
        const int hb = (nr + 63) / 64, nb = (nr + 255) / 256;  // row blocks of the chunk
        const int nh = sm.nhub, nitems = nh * hb + sm.nnorm * nb;
        for (;;) {
          int it = 0;
          if (lane == 0) it = atomicAdd(&sm.next, 1);
          it = __shfl_sync(0xffffffffu, it, 0);
          if (it >= nitems) break;
          const bool hub = it < nh * hb;
          const int c = hub ? sm.hubc[it / hb] : sm.normc[(it - nh * hb) / nb];
          const int rb = hub ? (it % hb) * 64 : ((it - nh * hb) % nb) * 256;
          const int deg = sm.cdeg[c], b0 = sm.cbeg[c];
          const int ds = max(0, min(deg, kPool - b0));  // pooled entries of the list
          const int rl = rb + (hub ? 2 * lane : 8 * lane);  // first row of the lane in the chunk
          const int i = r0 + rl;                            // even; a multiple of 4 for short lists
          if (hub) {
            float2 u = make_float2(0.f, 0.f);
            if (i < a.ldzt) {  // then i + 1 < ldzt
              const float* zt = a.ZTin + i;
              int q = 0;
              for (; q + 8 <= ds; q += 8) {
                float wt[8];
                float2 x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                  const int2 pe = sm.pool[b0 + q + t];
                  x[t] = __ldg(reinterpret_cast<const float2*>(zt + pe.x));
                  wt[t] = __int_as_float(pe.y);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                  u.x = fmaf(wt[t], x[t].x, u.x);
                  u.y = fmaf(wt[t], x[t].y, u.y);
                }
              }
              for (; q < ds; ++q) {
                const int2 pe = sm.pool[b0 + q];
                const float2 x = __ldg(reinterpret_cast<const float2*>(zt + pe.x));
                u.x = fmaf(__int_as_float(pe.y), x.x, u.x);
                u.y = fmaf(__int_as_float(pe.y), x.y, u.y);
              }
              for (int64_t f = sm.cf0[c] + ds; f < sm.cf0[c] + deg; ++f) {
                const int l = __ldg(a.Lc.col + f);
                const float w = __ldg(a.Lc.val + f);
                const float2 x =
                    __ldg(reinterpret_cast<const float2*>(a.ZTin + int64_t(a.inv ? a.inv[l] : l) * a.ldzt + i));
                u.x = fmaf(w, x.x, u.x);
                u.y = fmaf(w, x.y, u.y);
              }
            }
            sm.ac[c][rl] = u.x;
            sm.ac[c][rl + 1] = u.y;
          } else {
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
            if (i < a.ldzt) {  // then i + 3 < ldzt (both multiples of 4)
              const bool two = i + 4 < a.ldzt;  // then i + 7 < ldzt
              const float* zt = a.ZTin + i;
              int q = 0;
              for (; q + 4 <= ds; q += 4) {  // four neighbours' loads in flight
                float wt[4];
                float4 x[4], y[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  const int2 pe = sm.pool[b0 + q + t];
                  x[t] = ldg4(zt + pe.x);
                  y[t] = two ? ldg4(zt + pe.x + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                  wt[t] = __int_as_float(pe.y);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  fma4(u, wt[t], x[t]);
                  fma4(v, wt[t], y[t]);
                }
              }
              for (; q < ds; ++q) {
                const int2 pe = sm.pool[b0 + q];
                fma4(u, __int_as_float(pe.y), ldg4(zt + pe.x));
                if (two) fma4(v, __int_as_float(pe.y), ldg4(zt + pe.x + 4));
              }
              for (int64_t f = sm.cf0[c] + ds; f < sm.cf0[c] + deg; ++f) {
                const int l = __ldg(a.Lc.col + f);
                const float w = __ldg(a.Lc.val + f);
                const float* p = a.ZTin + int64_t(a.inv ? a.inv[l] : l) * a.ldzt + i;
                fma4(u, w, ldg4(p));
                if (two) fma4(v, w, ldg4(p + 4));
              }
            }
            *reinterpret_cast<float4*>(&sm.ac[c][rl]) = u;
            *reinterpret_cast<float4*>(&sm.ac[c][rl + 4]) = v;
          }
        }
      }
      if (!loaded) {  // the stripe's copy (overlapped with the first column pass)
        if (tid == 0 && !mbar_wait(&sm.mbar, k & 1, &sm.abort)) atomicExch(a.err, 1);
        loaded = true;
      }
      __syncthreads();  // sm.ac complete, the stripe in shared memory
      if (sm.abort) break;
      if (tid == 0) sm.next = 0;  // for the next chunk (after the barrier that ends this one)
      // ---- (Lr Z) from the stripe, prox, momentum: NQ lanes per row, lane
      // m of a row's group owning the quad of columns 4m .. 4m + 3 (the
      // group reads one contiguous 16 W-byte row of the stripe per entry)
      {
        const int m = tid % NQ, cq = 4 * m, jp = c0 + cq;
        const bool last = a.Pb && a.j == a.J;
        for (int rl = tid / NQ; rl < nr; rl += ST / NQ) {
          const int i = r0 + rl;
          const int f = rowp[i], d = rowp[i + 1] - f;
          const int32_t* lcol = a.Lr.col + rbase + f;
          const float* lval = a.Lr.val + rbase + f;
          float4 racc = make_float4(0.f, 0.f, 0.f, 0.f);
          int e = 0;
          for (; e + 8 <= d; e += 8) {  // eight entries' loads in flight
            int kk[8];
            float ww[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              kk[t] = __ldg(lcol + e + t);
              ww[t] = __ldg(lval + e + t);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) fma4(racc, ww[t], *reinterpret_cast<const float4*>(zs + kk[t] * W + cq));
          }
          for (; e < d; ++e)
            fma4(racc, __ldg(lval + e), *reinterpret_cast<const float4*>(zs + __ldg(lcol + e) * W + cq));
          const int64_t o = (int64_t(s) * a.rr + i) * W + cq;
          const float4 z4 = *reinterpret_cast<const float4*>(zs + i * W + cq);
          const float4 y4 = ldg4(a.Yb + o);
          const float4 s4 = *reinterpret_cast<const float4*>(a.Sb + o);
          float4 sv, zn;
          prox_entry(racc.x, sm.ac[cq][rl], z4.x, y4.x, s4.x, lam, a.two_gr, a.two_gc, a.mu, sv.x, zn.x);
          prox_entry(racc.y, sm.ac[cq + 1][rl], z4.y, y4.y, s4.y, lam, a.two_gr, a.two_gc, a.mu, sv.y, zn.y);
          prox_entry(racc.z, sm.ac[cq + 2][rl], z4.z, y4.z, s4.z, lam, a.two_gr, a.two_gc, a.mu, sv.z, zn.z);
          prox_entry(racc.w, sm.ac[cq + 3][rl], z4.w, y4.w, s4.w, lam, a.two_gr, a.two_gc, a.mu, sv.w, zn.w);
          if (last) *reinterpret_cast<float4*>(a.Pb + o) = s4;  // S_{J-1}
          *reinterpret_cast<float4*>(a.Sb + o) = sv;
          __stcg(reinterpret_cast<float4*>(a.Zout + o), zn);
          // Z_{j+1}^T: the groups of a warp write consecutive rows of a column
          float* zt = a.ZTout + int64_t(jp) * a.ldzt + i;
          if (jp < a.rc) zt[0] = zn.x;
          if (jp + 1 < a.rc) zt[a.ldzt] = zn.y;
          if (jp + 2 < a.rc) zt[2 * a.ldzt] = zn.z;
          if (jp + 3 < a.rc) zt[3 * a.ldzt] = zn.w;
          if (a.want_stats) {
            const float zz[4] = {z4.x, z4.y, z4.z, z4.w}, nn[4] = {zn.x, zn.y, zn.z, zn.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const double dd = double(nn[t]) - double(zz[t]);
              dz += dd * dd;
              nz += double(zz[t]) * double(zz[t]);
            }
          }
        }
      }
      __syncthreads();  // before the next chunk's sm.ac or the next stripe's copy
    }
    if (sm.abort) break;
    // every read of the buffer is done: load the next stripe into it
    if (tid == 0) {
      const int nx = int(gridDim.x + atomicAdd(a.ctr + a.j % 3, 1u));
      sm.next_stripe = nx;
      if (nx < a.nunits) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(nx);
      }
    }
    __syncthreads();
    u = sm.next_stripe;
  }
  if (sm.abort) {
    // the copy of stripe k may still be in flight: wait for it (bounded)
    // before the block leaves
    if (tid == 0) {
      int spare = 0;
      (void)mbar_wait(&sm.mbar, k & 1, &spare);
    }
    __syncthreads();
    return;
  }
  if (a.want_stats) {
    dz = warp_sum(dz);
    nz = warp_sum(nz);
    if (lane == 0) {
      sm.red[0][warp] = dz;
      sm.red[1][warp] = nz;
    }
    __syncthreads();
    if (tid == 0) {
      double sd = 0.0, sn = 0.0;
      for (int w = 0; w < ST / 32; ++w) {
        sd += sm.red[0][w];
        sn += sm.red[1][w];
      }
      atomicAdd(a.stats + 2 * (a.j & 3), sd);
      atomicAdd(a.stats + 2 * (a.j & 3) + 1, sn);
    }
  }
  if (a.j == a.J && blockIdx.x == 0 && tid == 0) a.done[1] = a.J;
}

// B (stripe-major, W columns per stripe, processing order) from A
// (row-major, ld lda): B[(s rr + i) W + c] = A[i, perm[s W + c]], zero past
// the last column.
template <int W>
__global__ void __launch_bounds__(256) to_stripes_kernel(const float* __restrict__ A, int64_t lda,
                                                         float* __restrict__ B, const int32_t* __restrict__ perm,
                                                         int rr, int rc, int nst) {
  const int64_t total = int64_t(nst) * rr * W;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t % W);
    const int64_t sr = t / W;
    const int i = int(sr % rr), q = int(sr / rr) * W + c;
    B[t] = q < rc ? A[int64_t(i) * lda + (perm ? perm[q] : q)] : 0.f;
  }
}

// A[i, perm[q]] = B[(s rr + i) W + c], q = s W + c < rc.
template <int W>
__global__ void __launch_bounds__(256) from_stripes_kernel(const float* __restrict__ B, float* __restrict__ A,
                                                           int64_t lda, const int32_t* __restrict__ perm, int rr,
                                                           int rc, int nst) {
  const int64_t total = int64_t(nst) * rr * W;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t % W);
    const int64_t sr = t / W;
    const int i = int(sr % rr), q = int(sr / rr) * W + c;
    if (q < rc) A[int64_t(i) * lda + (perm ? perm[q] : q)] = B[t];
  }
}

// Z_1 = S_0 = Y~ (cold start: S = Y~) or Z_{j0+1} = S_{j0} + mu_{j0}
// (S_{j0} - S_{j0-1}) (warm start, Sb holding S_{j0} and Pw S_{j0-1}), the
// operation the iteration applies; stripe-major into Zb and column-major
// into ZT0. The padding rows of both Z^T buffers are zeroed. A block takes
// 256 rows of one stripe and transposes them through shared memory.
template <int W>
__global__ void __launch_bounds__(256) stripe_init_kernel(const float* __restrict__ Yb, float* __restrict__ Sb,
                                                          const float* __restrict__ Pw, float mu0, int rr, int rc,
                                                          int nst, float* __restrict__ Zb, float* __restrict__ ZT0,
                                                          float* __restrict__ ZT1, int64_t ldzt) {
  __shared__ float tile[W][257];
  const int nrb = int((ldzt + 255) / 256);
  for (int64_t b = blockIdx.x; b < int64_t(nst) * nrb; b += gridDim.x) {
    const int s = int(b / nrb), i0 = int(b % nrb) * 256;
    for (int e = threadIdx.x; e < 256 * W; e += 256) {
      const int r = e / W, c = e % W, i = i0 + r;
      float z = 0.f;
      if (i < rr) {
        const int64_t o = (int64_t(s) * rr + i) * W + c;
        if (Pw) {
          const float sv = Sb[o], sp = Pw[o];
          z = fmaf(mu0, sv - sp, sv);
        } else {
          z = Yb[o];
          Sb[o] = z;
        }
        Zb[o] = z;
      }
      tile[c][r] = z;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 256 * W; e += 256) {
      const int c = e / 256, r = e % 256, i = i0 + r, q = s * W + c;
      if (q < rc && i < ldzt) {
        ZT0[int64_t(q) * ldzt + i] = tile[c][r];
        if (i >= rr) ZT1[int64_t(q) * ldzt + i] = 0.f;
      }
    }
    __syncthreads();
  }
}

template <int W>
size_t stripe_smem(int rr) {
  return smem_head<W>() + size_t(rr) * W * sizeof(float) + size_t(rr + 1) * sizeof(int32_t);
}

// Stripe width for rr rows: 16 when its stripe fits one block's shared
// memory, else 8, else 0 (not eligible). (Measured on the 2000 x 10000
// sampled matrix of the 8 GB workload: 433 us per iteration with W = 16,
// 484 us with W = 8 and two blocks per SM.)
int stripe_width(int rr) {
  const size_t cap = size_t(max_smem_optin());
  if (stripe_smem<16>(rr) <= cap) return 16;
  if (stripe_smem<8>(rr) <= cap) return 8;
  return 0;
}

template <int W>
cpca_status launch_to_stripes(const float* A, int64_t lda, float* B, const int32_t* perm, int rr, int rc,
                              cudaStream_t st) {
  const int nst = int(ceil_div(rc, W));
  const unsigned g = unsigned(std::min<int64_t>(ceil_div(int64_t(nst) * rr * W, 256), int64_t(num_sms()) * 8));
  to_stripes_kernel<W><<<g, 256, 0, st>>>(A, lda, B, perm, rr, rc, nst);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

template <int W>
cpca_status launch_from_stripes(const float* B, float* A, int64_t lda, const int32_t* perm, int rr, int rc,
                                cudaStream_t st) {
  const int nst = int(ceil_div(rc, W));
  const unsigned g = unsigned(std::min<int64_t>(ceil_div(int64_t(nst) * rr * W, 256), int64_t(num_sms()) * 8));
  from_stripes_kernel<W><<<g, 256, 0, st>>>(B, A, lda, perm, rr, rc, nst);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

template <int W>
cpca_status stripe_solve(const BatchProblem& P, const InstWs& iw, const StripeWs& sw, int J, double eps,
                         bool want_last, double t0, float mu0, int* err, cudaStream_t st) {
  const int rr = P.rr, rc = P.rc, nst = int(ceil_div(rc, W));
  const int64_t ldzt = (rr + 3) / 4 * 4;
  const int32_t* perm = nullptr;
  const int32_t* inv = nullptr;
  if (stripe_reorders(rr, rc)) {  // the column graph's locality order
    CPCA_TRY(graph_order(P.Lc, sw.perm, sw.inv, sw.oscr, sw.bar, err, st));
    perm = sw.perm;
    inv = sw.inv;
  }
  const bool warm = P.j0 > 0;
  CPCA_TRY(launch_to_stripes<W>(P.Yt, P.ldy, sw.Yb, perm, rr, rc, st));
  if (warm) {
    CPCA_TRY(launch_to_stripes<W>(P.X, P.ldx, sw.Sb, perm, rr, rc, st));
    CPCA_TRY(launch_to_stripes<W>(P.warm_prev, P.ldx, sw.Pb, perm, rr, rc, st));
  }
  CPCA_CUDA(cudaMemsetAsync(sw.ctr, 0, 3 * sizeof(unsigned int), st));  // stripe counters
  const int nrb = int(ceil_div(ldzt, 256));
  stripe_init_kernel<W><<<unsigned(std::min<int64_t>(int64_t(nst) * nrb, int64_t(num_sms()) * 8)), 256, 0, st>>>(
      sw.Yb, sw.Sb, warm ? sw.Pb : nullptr, mu0, rr, rc, nst, iw.Z0, iw.ZT0, iw.ZT1, ldzt);
  CPCA_LAUNCHED();
  const size_t smem = stripe_smem<W>(rr);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    return cudaFuncSetAttribute((const void*)fista_stripe_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(max_smem_optin()));
  }));
  StripeArgs a{};
  a.Yb = sw.Yb;
  a.Sb = sw.Sb;
  a.Pb = P.prev_out ? sw.Pb : nullptr;
  a.Lr = P.Lr;
  a.Lc = P.Lc;
  a.perm = perm;
  a.inv = inv;
  a.lam = iw.scal + 2;
  a.stats = iw.stats;
  a.done = iw.done;
  a.err = err;
  a.ctr = sw.ctr;
  a.ldzt = ldzt;
  a.two_gr = float(2.0 * P.gamma_r);
  a.two_gc = float(2.0 * P.gamma_c);
  a.rr = rr;
  a.rc = rc;
  a.nstripes = nst;
  {
    const int blocks = std::min(nst, Shape<W>::BLOCKS * num_sms());
    const int nhalf = rr >= 8 ? blocks : 0;  // the last wave's stripes, in halves
    a.nfull = nst - nhalf;
    a.nunits = a.nfull + 2 * nhalf;
  }
  a.J = J;
  a.eps = eps;
  const int grid = std::min(nst, Shape<W>::BLOCKS * num_sms());
  float* Z[2] = {iw.Z0, iw.Z1};
  float* ZT[2] = {iw.ZT0, iw.ZT1};
  double t = t0;  // t_{j0+j}; mu as in the constant-memory table of the resident kernel
  CPCA_PROF("fista_stripe", st);
  for (int j = 1; j <= J; ++j) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    a.mu = float((t - 1.0) / tn);
    t = tn;
    a.j = j;
    a.Zin = Z[(j - 1) & 1];
    a.ZTin = ZT[(j - 1) & 1];
    a.Zout = Z[j & 1];
    a.ZTout = ZT[j & 1];
    a.want_stats = (eps > 0 || (want_last && j == J)) ? 1 : 0;
    fista_stripe_kernel<W><<<grid, Shape<W>::ST, smem, st>>>(a);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      prof_end();
      set_error("striped FISTA launch: %s", cudaGetErrorString(e));
      return CPCA_ERR_CUDA;
    }
  }
  prof_end();
  CPCA_TRY(launch_from_stripes<W>(sw.Sb, P.X, P.ldx, perm, rr, rc, st));
  if (P.prev_out) CPCA_TRY(launch_from_stripes<W>(sw.Pb, P.prev_out, P.ldx, perm, rr, rc, st));
  return CPCA_OK;
}

}  // namespace

bool stripe_candidate(int rr, int rc) { return rr >= 64 && rr <= kStripeMaxRows && rc >= 256; }

size_t stripe_zcols(int rc) { return size_t(rc + 15) / 16 * 16; }

bool stripe_eligible(int rr, int rc) {
  if (!stripe_candidate(rr, rc)) return false;
  const int W = stripe_width(rr);
  // enough stripes to occupy the SMs; Z^T offsets below 2^31 (32-bit staged
  // offsets), as are Lr's row offsets (at most rr^2 entries)
  return W > 0 && ceil_div(rc, W) >= num_sms() && int64_t(rc) * ((rr + 3) / 4 * 4) < (int64_t(1) << 31);
}

bool stripe_reorders(int rr, int rc) { return int64_t(rr) * rc >= (int64_t(1) << 22) && order_supported(rc); }

StripeWs stripe_layout(Carve& c, int rr, int rc) {
  StripeWs w{};
  if (!stripe_candidate(rr, rc)) return w;
  const size_t n = size_t(rr) * stripe_zcols(rc);
  w.Yb = c.take<float>(n);
  w.Sb = c.take<float>(n);
  w.Pb = c.take<float>(n);
  w.perm = c.take<int32_t>(rc);
  w.inv = c.take<int32_t>(rc);
  w.oscr = c.take<unsigned char>(order_scratch_bytes(rc));
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  w.ctr = c.take<unsigned int>(3);
  return w;
}

cpca_status fista_stripe_run(const BatchProblem& P, const InstWs& iw, const StripeWs& sw, int J, double eps,
                             bool want_last, double t0, float mu0, int* err, cudaStream_t st) {
  CPCA_CHECK_ARG(sw.Yb != nullptr && stripe_eligible(P.rr, P.rc),
                 "frpcag: %d x %d problem outside the striped launch", P.rr, P.rc);
  return stripe_width(P.rr) == 16 ? stripe_solve<16>(P, iw, sw, J, eps, want_last, t0, mu0, err, st)
                                  : stripe_solve<8>(P, iw, sw, J, eps, want_last, t0, mu0, err, st);
}

}  // namespace cpca
