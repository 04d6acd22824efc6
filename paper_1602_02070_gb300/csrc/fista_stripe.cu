// fista_stripe.cu - FISTA for FRPCAG (Sec. IV-B, Algorithm 1) on single
// problems too large for the resident launch, one launch per iteration.
//
// The matrix is cut into stripes of SW = 8 columns spanning every row. A
// block takes stripes in turn; for each it brings the whole stripe of Z_j
// into shared memory with TMA (boxes of 8 columns x 256 rows, double-
// buffered: the next stripe's load runs while the current one computes).
// Then, in chunks of 512 rows:
//   (Z Lc)(i, j) = sum_l Lc[j, l] Z^T(l, i): for each of the stripe's
//       columns, the neighbour columns' rows of Z^T are read as 32-byte
//       vectors through L1 (the whole Z^T of the iteration is read-only
//       inside the launch);
//   (Lr Z)(i, j) = sum_k Lr[i, k] Z(k, j): entirely from the stripe in
//       shared memory (a row graph links arbitrary rows, and the stripe
//       holds all of them), 8 lanes per row;
//   S_j = prox(Z_j - lambda 2 (g_c Z Lc + g_r Lr Z)),
//   Z_{j+1} = S_j + mu_j (S_j - S_{j-1}),
// written row-major (S_j, Z_{j+1}) and column-major (Z_{j+1}^T, through
// shared memory for whole-row stores). Both graph sums run in CSR order
// with one FMA per entry, exactly as the resident kernel's: the iterates are
// bit for bit those of fista_batch_kernel. Launch boundaries order the
// iterations, so there is no grid barrier; with eps > 0 every launch first
// reads the previous iteration's statistics and all its blocks leave once
// the stopping test holds.
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
constexpr int SCHUNK = 512;    // rows per chunk
constexpr int STHREADS = 512;  // 16 warps
constexpr int SCN = 64;        // staged neighbour entries per stripe column

struct StripeArgs {
  CUtensorMap zmap;  // Z_j, row-major (ld ldz), boxes of SW x SBOX
  const float* ZTin;
  float* Zout;
  float* ZTout;
  const float* Yt;
  float* S;
  CsrView Lr, Lc;
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
  float zn[SW][SCHUNK];     // Z_{j+1} of the chunk, [column][row]
  int32_t coff[SW][SCN];    // neighbour column l -> element offset l * ldzt
  float cval[SW][SCN];
  int64_t cf0[SW];
  int cdeg[SW];
  uint64_t mbar[2];
  double red[2][STHREADS / 32];
  int abort;
};

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

__global__ void __launch_bounds__(STHREADS, 1) fista_stripe_kernel(const __grid_constant__ StripeArgs a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  StripeSmem& sm = *reinterpret_cast<StripeSmem*>(smraw);
  float* zs0 = reinterpret_cast<float*>(smraw + ((sizeof(StripeSmem) + 127) & ~size_t(127)));
  int32_t* rowp = reinterpret_cast<int32_t*>(zs0 + size_t(2) * a.rr_pad * SW);  // [rr + 1], from rowptr[0]
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
    mbar_init(&sm.mbar[1], 1);
    mbar_fence_init();
  }
  // row pointers of Lr relative to its first entry, for every stripe
  const int64_t rbase = a.Lr.rowptr[0];
  for (int i = tid; i <= a.rr; i += STHREADS) rowp[i] = int32_t(a.Lr.rowptr[i] - rbase);
  __syncthreads();
  auto issue = [&](int s, int buf) {  // one thread: the whole stripe s into buffer buf
    float* dst = zs0 + size_t(buf) * a.rr_pad * SW;
    mbar_expect_tx(&sm.mbar[buf], stripe_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_2d(dst + size_t(b) * SBOX * SW, &a.zmap, &sm.mbar[buf], s * SW, b * SBOX);
  };
  if (tid == 0) {
    if (int(blockIdx.x) < a.nstripes) issue(blockIdx.x, 0);
    if (int(blockIdx.x + gridDim.x) < a.nstripes) issue(blockIdx.x + gridDim.x, 1);
  }
  double dz = 0.0, nz = 0.0;
  int k = 0;
  for (int s = blockIdx.x; s < a.nstripes; s += gridDim.x, ++k) {
    const int buf = k & 1;
    const float* zs = zs0 + size_t(buf) * a.rr_pad * SW;
    const int c0 = s * SW;
    // neighbour lists of the stripe's columns (overlaps the stripe's load)
    if (tid < SW) {
      const int j = c0 + tid;
      const int64_t f0 = j < a.rc ? a.Lc.rowptr[j] : 0;
      sm.cf0[tid] = f0;
      sm.cdeg[tid] = j < a.rc ? int(a.Lc.rowptr[j + 1] - f0) : 0;
    }
    __syncthreads();
    for (int e = tid; e < SW * SCN; e += STHREADS) {
      const int c = e / SCN, q = e % SCN;
      if (q < min(sm.cdeg[c], SCN)) {
        sm.coff[c][q] = int32_t(__ldg(a.Lc.col + sm.cf0[c] + q)) * int32_t(a.ldzt);
        sm.cval[c][q] = __ldg(a.Lc.val + sm.cf0[c] + q);
      }
    }
    if (tid == 0 && !mbar_wait(&sm.mbar[buf], (k >> 1) & 1, &sm.abort)) atomicExch(a.err, 1);
    __syncthreads();
    if (sm.abort) break;
    for (int r0 = 0; r0 < a.rr; r0 += SCHUNK) {
      // ---- (Z Lc): warp -> stripe column c, 256-row half h; lane -> 8 rows
      {
        const int c = warp & (SW - 1), h = warp >> 3;
        const int rl = h * 256 + lane * 8, i = r0 + rl;
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
          for (int64_t f = sm.cf0[c] + SCN; f < sm.cf0[c] + deg; ++f)
            add(int64_t(__ldg(a.Lc.col + f)) * a.ldzt, __ldg(a.Lc.val + f));
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
            float zn = 0.f;
            if (jin) {
              const float z = zs[size_t(i) * SW + c];
              const float y = h ? yB : yA, sp = h ? spB : spA, acc = h ? accB : accA;
              const float gr = fmaf(a.two_gr, acc, a.two_gc * sm.ac[c][rl]);
              const float v = fmaf(-lam, gr, z);
              const float dl = v - y;
              const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
              zn = fmaf(a.mu, sv - sp, sv);
              if (a.prev_out && a.j == a.J) a.prev_out[int64_t(i) * a.lds + j] = sp;
              a.S[int64_t(i) * a.lds + j] = sv;
              a.Zout[int64_t(i) * a.ldz + j] = zn;
              if (a.want_stats) {
                const double d = double(zn) - double(z);
                dz += d * d;
                nz += double(z) * double(z);
              }
            }
            sm.zn[c][rl] = zn;
          }
        }
      }
      __syncthreads();
      // ---- Z_{j+1}^T: the chunk's rows of each stripe column, whole vectors
      {
        const int c = warp & (SW - 1), h = warp >> 3, j = c0 + c;
        const int rl = h * 256 + lane * 8, i = r0 + rl;
        if (j < a.rc && i < a.rr) {
          float* p = a.ZTout + int64_t(j) * a.ldzt + i;
          if (i + 8 <= a.rr) {
            *reinterpret_cast<float4*>(p) = *reinterpret_cast<const float4*>(&sm.zn[c][rl]);
            *reinterpret_cast<float4*>(p + 4) = *reinterpret_cast<const float4*>(&sm.zn[c][rl + 4]);
          } else {
            for (int t = 0; i + t < a.rr; ++t) p[t] = sm.zn[c][rl + t];
          }
        }
      }
      __syncthreads();
    }
    // every read of this buffer is done: load the stripe after next into it
    if (tid == 0 && s + 2 * int(gridDim.x) < a.nstripes) issue(s + 2 * gridDim.x, buf);
  }
  if (sm.abort) {
    // loads of stripes k and k + 1 may still be in flight: wait for them
    // (bounded) before the block leaves
    if (tid == 0)
      for (int d = 0; d < 2; ++d) {
        const int kk = k + d;
        if (int(blockIdx.x) + kk * int(gridDim.x) >= a.nstripes) continue;
        int spare = 0;
        (void)mbar_wait(&sm.mbar[kk & 1], (kk >> 1) & 1, &spare);
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

size_t stripe_smem(int rr_pad) {
  return ((sizeof(StripeSmem) + 127) & ~size_t(127)) + size_t(2) * rr_pad * SW * sizeof(float) +
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
  return stripe_smem(rr_pad) <= size_t(max_smem_optin()) && int64_t(rc) * ((rr + 3) / 4 * 4) < (int64_t(1) << 31) &&
         encode_fn() != nullptr;  // (Lr has at most rr^2 < 2^31 entries: 32-bit row offsets)
}

cpca_status fista_stripe_run(const BatchProblem& P, const InstWs& iw, int J, double eps, bool want_last,
                             double t0, int* err, cudaStream_t st) {
  const int rr = P.rr, rc = P.rc;
  const int rr_pad = int(ceil_div(rr, SBOX)) * SBOX;
  const int64_t ldz = (rc + 3) / 4 * 4, ldzt = (rr + 3) / 4 * 4;
  CUtensorMap maps[2];
  CPCA_CHECK_ARG(make_zmap(&maps[0], iw.Z0, rr, ldz) && make_zmap(&maps[1], iw.Z1, rr, ldz),
                 "frpcag: tensor map for the striped FISTA launch could not be encoded");
  const size_t smem = stripe_smem(rr_pad);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    return cudaFuncSetAttribute((const void*)fista_stripe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(max_smem_optin()));
  }));
  StripeArgs a{};
  a.Yt = P.Yt;
  a.S = P.X;
  a.Lr = P.Lr;
  a.Lc = P.Lc;
  a.lam = iw.scal + 2;
  a.stats = iw.stats;
  a.done = iw.done;
  a.err = err;
  a.ldy = P.ldy;
  a.lds = P.ldx;
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
  a.prev_out = P.prev_out;
  const int grid = std::min(a.nstripes, num_sms());
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
  return CPCA_OK;
}

}  // namespace cpca
