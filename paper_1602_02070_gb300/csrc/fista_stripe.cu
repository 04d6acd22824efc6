// fista_stripe.cu - FISTA for FRPCAG (Sec. IV-B, Algorithm 1) on single
// problems too large for the resident launch, one launch per iteration.
//
// The matrix is cut into stripes of SW = 8 columns spanning every row. A
// block (two per SM, so that one computes while the other waits for its
// stripe) takes stripes in turn; for each it brings the whole stripe of Z_j
// into shared memory with TMA (boxes of 8 columns x 256 rows). Then, in
// chunks of 256 rows:
//   (Z Lc)(i, j) = sum_l Lc[j, l] Z^T(l, i): a warp per stripe column, each
//       lane 8 consecutive rows, the neighbour columns' rows of Z^T read
//       through L1 as 32-byte vectors, eight neighbours in flight (the whole
//       Z^T of the iteration is read-only inside the launch);
//   (Lr Z)(i, j) = sum_k Lr[i, k] Z(k, j): entirely from the stripe in
//       shared memory (a row graph links arbitrary rows, and the stripe holds
//       all of them), 8 lanes per row, two rows per lane group at a time;
//   S_j = prox(Z_j - lambda 2 (g_c Z Lc + g_r Lr Z)),
//   Z_{j+1} = S_j + mu_j (S_j - S_{j-1}),
// written row-major (S_j, Z_{j+1}) and column-major (Z_{j+1}^T). Both graph
// sums run in CSR order with one FMA per entry, exactly as the resident
// kernel's: the iterates are bit for bit those of fista_batch_kernel.
// Launch boundaries order the iterations, so there is no grid barrier; with
// eps > 0 every launch first reads the previous iteration's statistics and
// all its blocks leave once the stopping test holds.
//
// Column order: for large problems the columns are processed in a
// locality order of the column graph (order.cu: components, then
// breadth-first levels), so that the stripes in flight gather their Z^T
// rows from a narrow band that stays in L2. Y~, S and the iterates are
// permuted into that order once per solve and X is permuted back at the
// end; each column keeps its CSR entry order, so the arithmetic - and the
// result - is unchanged.
//
// Algorithmic bytes per iteration: read Y~, S_{j-1}, Z_j (stripe), Z_j^T
// (gathers), write S_j, Z_{j+1}, Z_{j+1}^T: 28 B per entry when every
// gathered row comes from L2, plus the CSR bytes.
#include "fista_internal.cuh"
#include "tma.cuh"

namespace cpca {
namespace {

constexpr int SW = 8;          // stripe width (columns)
constexpr int SBOX = 256;      // rows per TMA box
constexpr int SCHUNK = 256;    // rows per chunk
constexpr int STHREADS = 256;  // 8 warps: a warp per stripe column in the column product
constexpr int SBLOCKS = 2;     // blocks per SM (one stripe buffer each)
constexpr int SCN = 64;        // staged neighbour entries per stripe column

struct StripeArgs {
  CUtensorMap zmap;  // Z_j, row-major (ld ldz), boxes of SW x SBOX
  const float* ZTin;
  float* Zout;
  float* ZTout;
  const float* Yt;
  float* S;
  CsrView Lr, Lc;
  const int32_t* perm;  // processing position -> column of Lc (null: identity)
  const int32_t* inv;   // column of Lc -> processing position
  const double* lam;
  double* stats;  // ring [4][2]
  int* done;      // [stopped, iterations]
  int* err;       // mbarrier timeout flag
  float* prev_out;  // S_{J-1} (ld lds) on the last iteration, or null
  int64_t ldy, lds, ldz, ldzt;
  float two_gr, two_gc, mu;
  int rr, rc, rr_pad, nstripes;
  int j, J;
  double eps;
  int want_stats;
};

struct StripeSmem {
  float ac[SW][SCHUNK];     // (Z Lc) of the chunk, [column][row]
  int32_t coff[SW][SCN];    // neighbour column -> element offset of its Z^T row
  float cval[SW][SCN];
  int64_t cf0[SW];
  int cdeg[SW];
  uint64_t mbar[1];
  double red[2][STHREADS / 32];
  int abort;
};

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

__global__ void __launch_bounds__(STHREADS, SBLOCKS) fista_stripe_kernel(const __grid_constant__ StripeArgs a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  StripeSmem& sm = *reinterpret_cast<StripeSmem*>(smraw);
  float* zs0 = reinterpret_cast<float*>(smraw + ((sizeof(StripeSmem) + 127) & ~size_t(127)));
  int32_t* rowp = reinterpret_cast<int32_t*>(zs0 + size_t(a.rr_pad) * SW);  // [rr + 1], from rowptr[0]
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
  const float lam = float(*a.lam);
  const int nbox = a.rr_pad / SBOX;
  const uint32_t stripe_bytes = uint32_t(a.rr_pad) * SW * 4;
  if (tid == 0) {
    sm.abort = 0;
    mbar_init(&sm.mbar[0], 1);
    mbar_fence_init();
  }
  // row pointers of Lr relative to its first entry, for every stripe
  const int64_t rbase = a.Lr.rowptr[0];
  for (int i = tid; i <= a.rr; i += STHREADS) rowp[i] = int32_t(a.Lr.rowptr[i] - rbase);
  __syncthreads();
  auto issue = [&](int s) {  // one thread: the whole stripe s into the buffer
    mbar_expect_tx(&sm.mbar[0], stripe_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_2d(zs0 + size_t(b) * SBOX * SW, &a.zmap, &sm.mbar[0], s * SW, b * SBOX);
  };
  if (tid == 0 && int(blockIdx.x) < a.nstripes) issue(blockIdx.x);
  double dz = 0.0, nz = 0.0;
  int k = 0;
  for (int s = blockIdx.x; s < a.nstripes; s += gridDim.x, ++k) {
    const float* zs = zs0;
    const int c0 = s * SW;
    // neighbour lists of the stripe's columns (overlaps the stripe's load)
    if (tid < SW) {
      const int jp = c0 + tid;
      const int jc = jp < a.rc ? (a.perm ? a.perm[jp] : jp) : 0;
      const int64_t f0 = jp < a.rc ? a.Lc.rowptr[jc] : 0;
      sm.cf0[tid] = f0;
      sm.cdeg[tid] = jp < a.rc ? int(a.Lc.rowptr[jc + 1] - f0) : 0;
    }
    __syncthreads();
    for (int e = tid; e < SW * SCN; e += STHREADS) {
      const int c = e / SCN, q = e % SCN;
      if (q < min(sm.cdeg[c], SCN)) {
        const int l = __ldg(a.Lc.col + sm.cf0[c] + q);
        sm.coff[c][q] = int32_t(a.inv ? a.inv[l] : l) * int32_t(a.ldzt);
        sm.cval[c][q] = __ldg(a.Lc.val + sm.cf0[c] + q);
      }
    }
    if (tid == 0 && !mbar_wait(&sm.mbar[0], k & 1, &sm.abort)) atomicExch(a.err, 1);
    __syncthreads();
    if (sm.abort) break;
    for (int r0 = 0; r0 < a.rr; r0 += SCHUNK) {
      // ---- (Z Lc): warp -> stripe column c, lane -> 8 consecutive rows
      {
        const int c = warp, rl = lane * 8, i = r0 + rl;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int deg = sm.cdeg[c];
        if (i < a.rr) {
          const bool full = i + 8 <= int(a.ldzt);
          const int ds = min(deg, SCN);
          auto add = [&](int64_t off, float w) {
            const float* p = a.ZTin + off + i;
            if (full) {
              const float4 u = ldg4(p), v = ldg4(p + 4);
              acc[0] = fmaf(w, u.x, acc[0]);
              acc[1] = fmaf(w, u.y, acc[1]);
              acc[2] = fmaf(w, u.z, acc[2]);
              acc[3] = fmaf(w, u.w, acc[3]);
              acc[4] = fmaf(w, v.x, acc[4]);
              acc[5] = fmaf(w, v.y, acc[5]);
              acc[6] = fmaf(w, v.z, acc[6]);
              acc[7] = fmaf(w, v.w, acc[7]);
            } else {
#pragma unroll
              for (int t = 0; t < 8; ++t)
                if (i + t < a.rr) acc[t] = fmaf(w, __ldg(p + t), acc[t]);
            }
          };
          int q = 0;
          if (full) {
            for (; q + 8 <= ds; q += 8) {  // eight neighbours' loads in flight
              float4 u[8], v[8];
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const float* p = a.ZTin + sm.coff[c][q + t] + i;
                u[t] = ldg4(p);
                v[t] = ldg4(p + 4);
              }
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const float w = sm.cval[c][q + t];
                acc[0] = fmaf(w, u[t].x, acc[0]);
                acc[1] = fmaf(w, u[t].y, acc[1]);
                acc[2] = fmaf(w, u[t].z, acc[2]);
                acc[3] = fmaf(w, u[t].w, acc[3]);
                acc[4] = fmaf(w, v[t].x, acc[4]);
                acc[5] = fmaf(w, v[t].y, acc[5]);
                acc[6] = fmaf(w, v[t].z, acc[6]);
                acc[7] = fmaf(w, v[t].w, acc[7]);
              }
            }
          }
          for (; q < ds; ++q) add(sm.coff[c][q], sm.cval[c][q]);
          for (int64_t f = sm.cf0[c] + SCN; f < sm.cf0[c] + deg; ++f) {
            const int l = __ldg(a.Lc.col + f);
            add(int64_t(a.inv ? a.inv[l] : l) * a.ldzt, __ldg(a.Lc.val + f));
          }
        }
        *reinterpret_cast<float4*>(&sm.ac[c][rl]) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        *reinterpret_cast<float4*>(&sm.ac[c][rl + 4]) = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      __syncthreads();
      // ---- (Lr Z) from the stripe, prox, momentum: 8 lanes per row, two
      // rows per lane group at a time (independent load chains), the row
      // pointers from shared memory, Y~ and S_{j-1} loaded up front
      {
        const int g = lane >> 3, c = lane & 7, j = c0 + c, gl = lane & ~7;
        const unsigned gmask = 0xFFu << gl;
        const bool jin = j < a.rc;
        for (int rA = warp * 4 + g; rA < SCHUNK; rA += 2 * (STHREADS / 8)) {
          const int rB = rA + STHREADS / 8;
          const int iA = r0 + rA, iB = r0 + rB;
          if (iA >= a.rr) break;  // uniform in the lane group
          const bool vB = rB < SCHUNK && iB < a.rr;
          float yA = 0.f, spA = 0.f, yB = 0.f, spB = 0.f;
          if (jin) {
            yA = __ldg(a.Yt + int64_t(iA) * a.ldy + j);
            spA = a.S[int64_t(iA) * a.lds + j];
            if (vB) {
              yB = __ldg(a.Yt + int64_t(iB) * a.ldy + j);
              spB = a.S[int64_t(iB) * a.lds + j];
            }
          }
          const int fA = rowp[iA], dA = rowp[iA + 1] - fA;
          const int fB = vB ? rowp[iB] : 0, dB = vB ? rowp[iB + 1] - fB : 0;
          float accA = 0.f, accB = 0.f;
          const int dmax = max(dA, dB);
          int kA = 0, kB = 0;
          float wA = 0.f, wB = 0.f;
          if (c < dA) { kA = __ldg(a.Lr.col + rbase + fA + c); wA = __ldg(a.Lr.val + rbase + fA + c); }
          if (c < dB) { kB = __ldg(a.Lr.col + rbase + fB + c); wB = __ldg(a.Lr.val + rbase + fB + c); }
          for (int e0 = 0; e0 < dmax; e0 += 8) {
            // the next eight entries of both rows, in flight during this step
            const int e1 = e0 + 8 + c;
            int nkA = 0, nkB = 0;
            float nwA = 0.f, nwB = 0.f;
            if (e1 < dA) { nkA = __ldg(a.Lr.col + rbase + fA + e1); nwA = __ldg(a.Lr.val + rbase + fA + e1); }
            if (e1 < dB) { nkB = __ldg(a.Lr.col + rbase + fB + e1); nwB = __ldg(a.Lr.val + rbase + fB + e1); }
            const int nA = min(8, dA - e0), nB = min(8, dB - e0);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int k1 = __shfl_sync(gmask, kA, gl + t), k2 = __shfl_sync(gmask, kB, gl + t);
              const float w1 = __shfl_sync(gmask, wA, gl + t), w2 = __shfl_sync(gmask, wB, gl + t);
              if (t < nA) accA = fmaf(w1, zs[size_t(k1) * SW + c], accA);
              if (t < nB) accB = fmaf(w2, zs[size_t(k2) * SW + c], accB);
            }
            kA = nkA; wA = nwA; kB = nkB; wB = nwB;
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int rl = h ? rB : rA, i = h ? iB : iA;
            if (h && !vB) break;
            if (jin) {
              const float z = zs[size_t(i) * SW + c];
              const float y = h ? yB : yA, sp = h ? spB : spA, acc = h ? accB : accA;
              const float gr = fmaf(a.two_gr, acc, a.two_gc * sm.ac[c][rl]);
              const float v = fmaf(-lam, gr, z);
              const float dl = v - y;
              const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
              const float zn = fmaf(a.mu, sv - sp, sv);
              if (a.prev_out && a.j == a.J) a.prev_out[int64_t(i) * a.lds + j] = sp;
              a.S[int64_t(i) * a.lds + j] = sv;
              a.Zout[int64_t(i) * a.ldz + j] = zn;
              // Z_{j+1}^T: the four row groups of a warp fill 16 consecutive
              // bytes of each of the stripe's rows of Z^T
              a.ZTout[int64_t(j) * a.ldzt + i] = zn;
              if (a.want_stats) {
                const double d = double(zn) - double(z);
                dz += d * d;
                nz += double(z) * double(z);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    // every read of the buffer is done: load the next stripe into it
    if (tid == 0 && s + int(gridDim.x) < a.nstripes) issue(s + gridDim.x);
  }
  if (sm.abort) {
    // the load of stripe k may still be in flight: wait for it (bounded)
    // before the block leaves
    if (tid == 0) {
      int spare = 0;
      (void)mbar_wait(&sm.mbar[0], k & 1, &spare);
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
      for (int w = 0; w < STHREADS / 32; ++w) {
        sd += sm.red[0][w];
        sn += sm.red[1][w];
      }
      atomicAdd(a.stats + 2 * (a.j & 3), sd);
      atomicAdd(a.stats + 2 * (a.j & 3) + 1, sn);
    }
  }
  if (a.j == a.J && blockIdx.x == 0 && tid == 0) a.done[1] = a.J;
}

// Z_1 = S_0 = Y~ (cold start) or Z_{j0+1} = S_{j0} + mu_{j0} (S_{j0} -
// S_{j0-1}) (warm start, S holding S_{j0}), written row-major and as Z^T;
// the padding columns of Z and rows of Z^T (both buffers) are zeroed.
__global__ void __launch_bounds__(256)
stripe_init_kernel(const float* __restrict__ Yt, int64_t ldy, float* __restrict__ S, int64_t lds,
                   const float* __restrict__ warm_prev, float mu0, int rr, int rc, float* __restrict__ Z0,
                   float* __restrict__ Z1, float* __restrict__ ZT0, float* __restrict__ ZT1, int64_t ldz,
                   int64_t ldzt) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int nti = int((ldzt + 31) / 32), ntc = int((ldz + 31) / 32);
  for (int64_t t = blockIdx.x; t < int64_t(nti) * ntc; t += gridDim.x) {
    const int i0 = int(t / ntc) * 32, j0 = int(t % ntc) * 32;
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, j = j0 + tx;
      float z = 0.f;
      if (i < rr && j < rc) {
        if (warm_prev) {
          const float sv = S[int64_t(i) * lds + j], sp = warm_prev[int64_t(i) * lds + j];
          z = fmaf(mu0, sv - sp, sv);
        } else {
          z = Yt[int64_t(i) * ldy + j];
          S[int64_t(i) * lds + j] = z;
        }
      }
      if (i < rr && j < ldz) {
        Z0[int64_t(i) * ldz + j] = z;
        Z1[int64_t(i) * ldz + j] = 0.f;
      }
      tile[r][tx] = z;
    }
    __syncthreads();
    for (int c = ty; c < 32; c += 8) {
      const int j = j0 + c, i = i0 + tx;
      if (j < rc && i < ldzt) {
        ZT0[int64_t(j) * ldzt + i] = tile[tx][c];
        ZT1[int64_t(j) * ldzt + i] = 0.f;
      }
    }
    __syncthreads();
  }
}

// B(:, q) = A(:, perm[q]) (forward) or B(:, perm[q]) = A(:, q) (backward),
// `rows` rows of `cols` columns.
__global__ void permute_cols_kernel(const float* __restrict__ A, int64_t lda, float* __restrict__ B, int64_t ldb,
                                    const int32_t* __restrict__ perm, int rows, int cols, int backward) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < int64_t(rows) * cols;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / cols), q = int(t % cols);
    if (backward)
      B[int64_t(i) * ldb + perm[q]] = A[int64_t(i) * lda + q];
    else
      B[int64_t(i) * ldb + q] = A[int64_t(i) * lda + perm[q]];
  }
}

size_t stripe_smem(int rr_pad) {
  return ((sizeof(StripeSmem) + 127) & ~size_t(127)) + size_t(rr_pad) * SW * sizeof(float) +
         size_t(rr_pad + 1) * sizeof(int32_t);
}

bool make_zmap(CUtensorMap* map, const float* Z, int rr, int64_t ldz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(ldz), cuuint64_t(rr)};
  cuuint64_t strides[1] = {cuuint64_t(ldz) * 4};
  cuuint32_t box[2] = {cuuint32_t(SW), cuuint32_t(SBOX)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Z), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool stripe_eligible(int rr, int rc) {
  if (rr < SBOX || rc < 4 * SW) return false;
  const int rr_pad = int(ceil_div(rr, SBOX)) * SBOX;
  // (Lr has at most rr^2 < 2^31 entries: 32-bit row offsets)
  return stripe_smem(rr_pad) <= size_t(max_smem_optin()) / SBLOCKS && int64_t(rc) * ((rr + 3) / 4 * 4) < (int64_t(1) << 31) &&
         encode_fn() != nullptr;
}

bool stripe_reorders(int rr, int rc) {
  return rr >= SBOX && rc >= 4 * SW && int64_t(rr) * rc >= (int64_t(1) << 22) && order_supported(rc);
}

StripeWs stripe_layout(Carve& c, int rr, int rc) {
  StripeWs w{};
  if (!stripe_reorders(rr, rc)) return w;
  const size_t ldz = size_t(rc + 3) / 4 * 4;
  w.Yp = c.take<float>(size_t(rr) * ldz);
  w.Sp = c.take<float>(size_t(rr) * ldz);
  w.Pp = c.take<float>(size_t(rr) * ldz);
  w.perm = c.take<int32_t>(rc);
  w.inv = c.take<int32_t>(rc);
  w.oscr = c.take<unsigned char>(order_scratch_bytes(rc));
  w.bar = c.take<unsigned int>(kBarrierCounters + 1);
  return w;
}

cpca_status fista_stripe_run(const BatchProblem& P, const InstWs& iw, const StripeWs& sw, int J, double eps,
                             bool want_last, double t0, float mu0, int* err, cudaStream_t st) {
  const int rr = P.rr, rc = P.rc;
  const int rr_pad = int(ceil_div(rr, SBOX)) * SBOX;
  const int64_t ldz = (rc + 3) / 4 * 4, ldzt = (rr + 3) / 4 * 4;
  CUtensorMap maps[2];
  CPCA_CHECK_ARG(make_zmap(&maps[0], iw.Z0, rr, ldz) && make_zmap(&maps[1], iw.Z1, rr, ldz),
                 "frpcag: tensor map for the striped FISTA launch could not be encoded");
  // locality order of the columns (large problems with the ordering scratch)
  const bool reorder = sw.Yp != nullptr;
  const float* Y = P.Yt;
  float* S = P.X;
  int64_t ldy = P.ldy, lds = P.ldx;
  const float* warm = P.j0 > 0 ? P.warm_prev : nullptr;
  float* prev = P.prev_out;
  const unsigned pg = std::min<unsigned>(ceil_div(int64_t(rr) * rc, 256), num_sms() * 8);
  if (reorder) {
    CPCA_TRY(graph_order(P.Lc, sw.perm, sw.inv, sw.oscr, sw.bar, err, st));
    permute_cols_kernel<<<pg, 256, 0, st>>>(P.Yt, P.ldy, sw.Yp, ldz, sw.perm, rr, rc, 0);
    CPCA_LAUNCHED();
    if (warm) {
      permute_cols_kernel<<<pg, 256, 0, st>>>(P.X, P.ldx, sw.Sp, ldz, sw.perm, rr, rc, 0);
      CPCA_LAUNCHED();
      permute_cols_kernel<<<pg, 256, 0, st>>>(warm, P.ldx, sw.Pp, ldz, sw.perm, rr, rc, 0);
      CPCA_LAUNCHED();
      warm = sw.Pp;
    }
    Y = sw.Yp;
    S = sw.Sp;
    ldy = lds = ldz;
    if (prev) prev = sw.Pp;
  }
  stripe_init_kernel<<<std::min<unsigned>(ceil_div(int64_t(rr) * ldz, 1024), num_sms() * 8), 256, 0, st>>>(
      Y, ldy, S, lds, warm, mu0, rr, rc, iw.Z0, iw.Z1, iw.ZT0, iw.ZT1, ldz, ldzt);
  CPCA_LAUNCHED();
  const size_t smem = stripe_smem(rr_pad);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    return cudaFuncSetAttribute((const void*)fista_stripe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(max_smem_optin() / SBLOCKS));
  }));
  StripeArgs a{};
  a.Yt = Y;
  a.S = S;
  a.Lr = P.Lr;
  a.Lc = P.Lc;
  a.perm = reorder ? sw.perm : nullptr;
  a.inv = reorder ? sw.inv : nullptr;
  a.lam = iw.scal + 2;
  a.stats = iw.stats;
  a.done = iw.done;
  a.err = err;
  a.prev_out = prev;
  a.ldy = ldy;
  a.lds = lds;
  a.ldz = ldz;
  a.ldzt = ldzt;
  a.two_gr = float(2.0 * P.gamma_r);
  a.two_gc = float(2.0 * P.gamma_c);
  a.rr = rr;
  a.rc = rc;
  a.rr_pad = rr_pad;
  a.nstripes = int(ceil_div(rc, SW));
  a.J = J;
  a.eps = eps;
  const int grid = std::min(a.nstripes, SBLOCKS * num_sms());
  float* Z[2] = {iw.Z0, iw.Z1};
  float* ZT[2] = {iw.ZT0, iw.ZT1};
  double t = t0;  // t_{j0+j}; mu as in the constant-memory table of the resident kernel
  CPCA_PROF("fista_stripe", st);
  for (int j = 1; j <= J; ++j) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    a.mu = float((t - 1.0) / tn);
    t = tn;
    a.j = j;
    a.zmap = maps[(j - 1) & 1];
    a.ZTin = ZT[(j - 1) & 1];
    a.Zout = Z[j & 1];
    a.ZTout = ZT[j & 1];
    a.want_stats = (eps > 0 || (want_last && j == J)) ? 1 : 0;
    fista_stripe_kernel<<<grid, STHREADS, smem, st>>>(a);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      prof_end();
      set_error("striped FISTA launch: %s", cudaGetErrorString(e));
      return CPCA_ERR_CUDA;
    }
  }
  prof_end();
  if (reorder) {
    permute_cols_kernel<<<pg, 256, 0, st>>>(sw.Sp, ldz, P.X, P.ldx, sw.perm, rr, rc, 1);
    CPCA_LAUNCHED();
    if (P.prev_out) {
      permute_cols_kernel<<<pg, 256, 0, st>>>(sw.Pp, ldz, P.prev_out, P.ldx, sw.perm, rr, rc, 1);
      CPCA_LAUNCHED();
    }
  }
  return CPCA_OK;
}

}  // namespace cpca
