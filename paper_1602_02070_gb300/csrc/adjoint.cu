// adjoint.cu - reverse-mode derivative of the FISTA solve (Algorithm 1 with
// a fixed iteration count, Sec. IV-B), of its step size lambda = 1/beta'
// (power iterations on both Laplacians), and of the Laplacians as functions
// of the edge weights (Sec. I). The paper has no derivatives: what is
// differentiated is the computed map, so that finite differences of
// cpca_frpcag_solve agree with it.
//
// Forward map, for j = 1..J (Z_1 = S_0 = Y~, t_1 = 1):
//   G_j = 2 gamma_r Lr Z_j + 2 gamma_c Z_j Lc,  R_j = Z_j - lambda G_j - Y~,
//   S_j = Y~ + sgn(R_j) max(|R_j| - lambda, 0),
//   Z_{j+1} = (1 + mu_j) S_j - mu_j S_{j-1},   mu_j = (t_j - 1) / t_{j+1}.
// Reverse, j = J..1, with Sb = dloss/dS_j and M_j = [|R_j| > lambda]:
//   Vb = M_j o Sb;  dY~ += Sb - Vb;
//   dlambda += -sum sgn(R_j) Vb - <Vb, G_j>;
//   dgamma_r += -2 lambda <Vb, Lr Z_j>;  dgamma_c += -2 lambda <Vb, Z_j Lc>;
//   dLr(a,b) += -2 lambda gamma_r sum_c Vb(a,c) Z_j(b,c)   (on Lr's pattern)
//   dLc(a,b) += -2 lambda gamma_c sum_r Z_j(r,a) Vb(r,b)   (on Lc's pattern)
//   Zb = Vb - lambda (2 gamma_r Lr Vb + 2 gamma_c Vb Lc)    (L symmetric)
//   dS_{j-1} += (1 + mu_{j-1}) Zb, dS_{j-2} += -mu_{j-1} Zb  (j >= 2)
//   dY~ += Zb + dS_0                                         (j = 1).
//
// Checkpointing: a first forward pass stores (S_j, Z_{j+1}) every C
// iterations; then, segment by segment from the last, the forward iterations
// of the segment are recomputed with every Z_j kept (row-major and
// column-major), and the reverse sweep runs over them. Both sweeps are
// persistent cooperative launches over 32 x 32 tiles with one grid barrier
// per iteration (two phases per reverse iteration: the mask phase publishes
// Vb, the second phase gathers Vb's neighbours). The derivatives with
// respect to the Laplacian entries are summed per tile column (Lr) and per
// tile row (Lc) in FP64 without atomics, then reduced in a fixed order.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fista_internal.cuh"

namespace cpca {
namespace {

// ------------------------------------------------------------- momentum --
// mu[j] = (t_j - 1) / t_{j+1} in the same double arithmetic as the solve.
__global__ void mu_kernel(int J, float* mu) {
  if (threadIdx.x || blockIdx.x) return;
  double t = 1.0;
  mu[0] = 0.f;
  for (int j = 1; j <= J; ++j) {
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    mu[j] = float((t - 1.0) / tn);
    t = tn;
  }
}

// Seed trajectory slot 0: Z (row-major, ld ldz, and its transpose, ld
// ldzt) and S (ld ldz) from Zsrc (ld lzs) and Ssrc (ld lss); the padding of
// the rows is zeroed.
__global__ void __launch_bounds__(256)
seed_kernel(const float* __restrict__ Zsrc, int64_t lzs, const float* __restrict__ Ssrc, int64_t lss, int rr,
            int rc, int64_t ldz, int64_t ldzt, float* __restrict__ Z, float* __restrict__ ZT,
            float* __restrict__ S) {
  __shared__ float tile[TB][TB + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntj = (rc + TB - 1) / TB, ntiles = ((rr + TB - 1) / TB) * ntj;
  for (int tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int i0 = (tl / ntj) * TB, j0 = (tl % ntj) * TB;
    const int ni = min(TB, rr - i0), nj = min(TB, rc - j0);
    for (int r = warp; r < TB; r += 8) {
      const int64_t i = i0 + r, jj = j0 + lane;
      const bool in = r < ni && lane < nj;
      const float z = in ? Zsrc[i * lzs + jj] : 0.f;
      if (r < ni && jj < ldz) {
        Z[i * ldz + jj] = z;
        S[i * ldz + jj] = in ? Ssrc[i * lss + jj] : 0.f;
      }
      tile[r][lane] = z;
    }
    __syncthreads();
    for (int c = warp; c < TB; c += 8)
      if (c < nj && i0 + lane < ldzt) ZT[int64_t(j0 + c) * ldzt + i0 + lane] = tile[lane][c];
    __syncthreads();
  }
}

struct TrajArgs {
  const float* Yt;
  int64_t ldy;
  int rr, rc, ntj, ntiles;
  int64_t ldz, ldzt;     // padded row lengths of the row- and column-major buffers
  int yvec, dyvec;       // Y~ / dY~ rows allow 16-byte accesses
  CsrView Lr, Lc;
  const double* lam;
  float two_gr, two_gc;
  double gamma_r, gamma_c;
  const float* mu;
  float* S;              // own tiles: S_{j-1} in, S_j out (ld ldz)
  float* Zs;             // trajectory slots of Z_j (row-major, slot stride rr * ldz)
  float* ZTs;            // column-major copies (slot stride rc * ldzt)
  uint8_t* Ms;           // step j's prox codes in the slot of Z_j (slot stride rr * ldz);
                         // bit 0: |V_j - Y~| > lambda, bit 1: V_j - Y~ < 0. Null: not kept
  int jbase, nslot;      // Z_j lives in slot (j - jbase) % nslot
  int ja, jb;            // forward: iterations ja..jb; reverse: jb down to ja
  int J;
  // forward only: checkpoints (S_j, Z_{j+1}) at j = m * ck, m = 1..
  float* ckS;
  float* ckZ;
  int ck;
  // reverse only
  float* Sb;             // dloss/dS_j (own tiles, ld ldz)
  float* A2;             // partial dloss/dS_{j-1}
  float* Vb[2];          // published Vb, row-major / column-major, parity j & 1
  float* VbT[2];
  float* dY;
  int64_t lddy;
  double* Pr;            // [ntj][nnz_r]
  double* Pc;            // [nti][nnz_c]
  double* scal_bar;      // [3]: dlambda, dgamma_r, dgamma_c (FP64 atomics)
  const int64_t* tmap_c; // index of entry (j, i) for each entry (i, j) of Lc
  GridBar bar;
};

__device__ __forceinline__ int slot_of(const TrajArgs& a, int j) {
  int s = (j - a.jbase) % a.nslot;
  return s < 0 ? s + a.nslot : s;
}
__device__ __forceinline__ float* zslot(const TrajArgs& a, int j) {
  return a.Zs + size_t(slot_of(a, j)) * size_t(a.rr) * size_t(a.ldz);
}
__device__ __forceinline__ float* ztslot(const TrajArgs& a, int j) {
  return a.ZTs + size_t(slot_of(a, j)) * size_t(a.rc) * size_t(a.ldzt);
}
__device__ __forceinline__ uint8_t* mslot(const TrajArgs& a, int j) {
  return a.Ms + size_t(slot_of(a, j)) * size_t(a.rr) * size_t(a.ldz);
}

__device__ __forceinline__ void tile_of(const TrajArgs& a, int tile, int& i0, int& j0, int& ni, int& nj) {
  i0 = (tile / a.ntj) * TB;
  j0 = (tile % a.ntj) * TB;
  ni = min(TB, a.rr - i0);
  nj = min(TB, a.rc - j0);
}

__device__ __forceinline__ float4 ld4(const float* p, bool vec, int n) {
  if (vec) return *reinterpret_cast<const float4*>(p);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (n > 0) v.x = p[0];
  if (n > 1) v.y = p[1];
  if (n > 2) v.z = p[2];
  if (n > 3) v.w = p[3];
  return v;
}
__device__ __forceinline__ void st4(float* p, float4 v, bool vec, int n) {
  if (vec) {
    *reinterpret_cast<float4*>(p) = v;
    return;
  }
  if (n > 0) p[0] = v.x;
  if (n > 1) p[1] = v.y;
  if (n > 2) p[2] = v.z;
  if (n > 3) p[3] = v.w;
}
__device__ __forceinline__ float& cmp(float4& v, int t) {
  return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}
__device__ __forceinline__ float cmp(const float4& v, int t) {
  return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

template <typename Off>
struct TrajSmem {
  TileNbrT<Off> nb;
  float ac[TB][TB + 1];
  float tl[TB][TB + 1];
  float pr[TB][kTileNbr];  // resident reverse: dL partial sums of the staged entries
  float pc[TB][kTileNbr];
};

// Forward iterations ja..jb with the trajectory kept: the solve's FISTA
// step, entry for entry, in its thread layout (lane group g of warp w owns
// tile row / column 4 w + g, each lane 4 consecutive entries). RESIDENT:
// one tile per block for the whole launch, lists staged once and S kept in
// registers (written back at the end); otherwise blocks stream over tiles.
template <bool RESIDENT>
__global__ void __launch_bounds__(256, RESIDENT ? 5 : 4)
traj_forward_kernel(const __grid_constant__ TrajArgs a) {
  using Off = typename std::conditional<RESIDENT, int32_t, int64_t>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  TrajSmem<Off>& sm = *reinterpret_cast<TrajSmem<Off>*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = warp * 4 + (lane >> 3), cq = 4 * (lane & 7);
  const float lam = float(*a.lam);
  float4 rs = make_float4(0.f, 0.f, 0.f, 0.f);
  if (RESIDENT) {
    int i0, j0, ni, nj;
    tile_of(a, blockIdx.x, i0, j0, ni, nj);
    stage_nbr(sm.nb, a.Lr, a.Lc, int(a.ldzt), int(a.ldz), i0, j0, ni, nj);
    if (rl < ni && cq < nj) rs = *reinterpret_cast<const float4*>(a.S + int64_t(i0 + rl) * a.ldz + j0 + cq);
  }
  for (int j = a.ja; j <= a.jb; ++j) {
    const float mu = a.mu[j];
    const float* Zin = zslot(a, j);
    const float* ZTin = ztslot(a, j);
    float* Zout = zslot(a, j + 1);
    float* ZTout = ztslot(a, j + 1);
    const bool ckpt = a.ck > 0 && j % a.ck == 0 && j < a.J;
    const size_t ckoff = ckpt ? size_t(j / a.ck - 1) * size_t(a.rr) * size_t(a.ldz) : 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      int i0, j0, ni, nj;
      tile_of(a, tile, i0, j0, ni, nj);
      if (!RESIDENT) stage_nbr(sm.nb, a.Lr, a.Lc, int(a.ldzt), int(a.ldz), i0, j0, ni, nj);
      {
        const float4 o = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.coff[rl], sm.nb.cval[rl], sm.nb.cdeg[rl],
                                                           sm.nb.cf0[rl], rl < nj && cq < ni, ZTin, i0 + cq,
                                                           a.Lc, a.ldzt);
        sm.ac[cq][rl] = o.x;
        sm.ac[cq + 1][rl] = o.y;
        sm.ac[cq + 2][rl] = o.z;
        sm.ac[cq + 3][rl] = o.w;
      }
      const bool own = rl < ni && cq < nj;
      float4 ar = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.roff[rl], sm.nb.rval[rl], sm.nb.rdeg[rl],
                                                    sm.nb.rf0[rl], own, Zin, j0 + cq, a.Lr, a.ldz);
      __syncthreads();
      float4 zn4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (own) {
        const int64_t i = i0 + rl, jj = j0 + cq;
        const int nv = nj - cq;
        float4 z4 = __ldcg(reinterpret_cast<const float4*>(Zin + i * a.ldz + jj));
        float4 y4 = ld4(a.Yt + i * a.ldy + jj, a.yvec, nv);
        float4 s4 = RESIDENT ? rs : *reinterpret_cast<const float4*>(a.S + i * a.ldz + jj);
        float4 sv4 = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t code = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q < nv) {
            const float z = cmp(z4, q), y = cmp(y4, q), sp = cmp(s4, q);
            const float gr = fmaf(a.two_gr, cmp(ar, q), a.two_gc * sm.ac[rl][cq + q]);
            const float v = fmaf(-lam, gr, z);
            const float dl = v - y;
            const float sv = y + copysignf(fmaxf(fabsf(dl) - lam, 0.f), dl);
            cmp(sv4, q) = sv;
            cmp(zn4, q) = fmaf(mu, sv - sp, sv);
            code |= uint32_t((fabsf(dl) - lam > 0.f ? 1 : 0) | (dl < 0.f ? 2 : 0)) << (8 * q);
          }
        }
        if (a.Ms) *reinterpret_cast<uint32_t*>(mslot(a, j) + i * a.ldz + jj) = code;
        if (RESIDENT) rs = sv4;
        else *reinterpret_cast<float4*>(a.S + i * a.ldz + jj) = sv4;
        *reinterpret_cast<float4*>(Zout + i * a.ldz + jj) = zn4;
        if (ckpt) {
          *reinterpret_cast<float4*>(a.ckS + ckoff + i * a.ldz + jj) = sv4;
          *reinterpret_cast<float4*>(a.ckZ + ckoff + i * a.ldz + jj) = zn4;
        }
      }
      sm.tl[rl][cq] = zn4.x;
      sm.tl[rl][cq + 1] = zn4.y;
      sm.tl[rl][cq + 2] = zn4.z;
      sm.tl[rl][cq + 3] = zn4.w;
      __syncthreads();
      if (rl < nj && cq < ni)
        *reinterpret_cast<float4*>(ZTout + int64_t(j0 + rl) * a.ldzt + i0 + cq) =
            make_float4(sm.tl[cq][rl], sm.tl[cq + 1][rl], sm.tl[cq + 2][rl], sm.tl[cq + 3][rl]);
      if (!RESIDENT) __syncthreads();
    }
    if (!grid_sync(a.bar)) return;
  }
  if (RESIDENT) {
    int i0, j0, ni, nj;
    tile_of(a, blockIdx.x, i0, j0, ni, nj);
    if (rl < ni && cq < nj) *reinterpret_cast<float4*>(a.S + int64_t(i0 + rl) * a.ldz + j0 + cq) = rs;
  }
}

// Partial sums of dL on the staged list `rl` of the tile (one list per
// 8-lane group; each lane holds 4 consecutive elements of the list's
// vectors): for every entry q, sum over the group of dot(x[off[q] + base],
// own) with x read as 16-byte vectors. Eight entries at a time: eight
// gathers per lane, then a butterfly over the group's 8 lanes (7 shuffles
// for 8 sums) after which every lane holds one entry's sum. The sums are
// added to acc[rl][q] (resident kernel, staged entries) or, times scale, to
// P at entry f0 + q (or its transpose tmap[f0 + q]). The loop bound is the
// warp's largest list so that all lanes take part in the shuffles.
template <bool RESIDENT, typename Off>
__device__ __forceinline__ void list_partials(const Off* off, int deg, int64_t f0, bool valid,
                                              const float* __restrict__ x, int64_t base, const CsrView& L,
                                              int64_t stride, float4 own, float* acc, double scale,
                                              double* __restrict__ P, const int64_t* __restrict__ tmap,
                                              int lane) {
  const int l8 = lane & 7;
  const bool h4 = l8 & 4, h2 = l8 & 2, h1 = l8 & 1;
  const int mine = (h4 ? 4 : 0) + (h2 ? 2 : 0) + (h1 ? 1 : 0);
  int dmax = deg;
  dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, 8));
  dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, 16));
  for (int q0 = 0; q0 < dmax; q0 += 8) {
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = q0 + t;
      float d = 0.f;
      if (valid && q < deg) {
        const int64_t o = q < kTileNbr ? int64_t(off[q]) : int64_t(__ldg(L.col + f0 + q)) * stride;
        d = dot4(__ldcg(reinterpret_cast<const float4*>(x + o + base)), own);
      }
      v[t] = d;
    }
    float w4[4], w2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = h4 ? v[i] : v[i + 4];
      const float keep = h4 ? v[i + 4] : v[i];
      w4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = h2 ? w4[i] : w4[i + 2];
      const float keep = h2 ? w4[i + 2] : w4[i];
      w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    const float send = h1 ? w2[0] : w2[1];
    const float keep = h1 ? w2[1] : w2[0];
    const float y = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    const int q = q0 + mine;
    if (q < deg && y != 0.f) {
      if (RESIDENT && q < kTileNbr) {
        acc[q] += y;
      } else {
        const int64_t e = f0 + q;
        const int64_t t = tmap ? __ldg(tmap + e) : e;  // -1: no transposed entry
        if (t >= 0) P[t] += scale * double(y);
      }
    }
  }
}

// Reverse iterations jb down to ja over the trajectory slots, one grid
// barrier per iteration. Entering iteration j, Vb_j = M_j o Sb_j is
// published in both layouts (M_j: step j's prox mask, kept by the forward).
// Iteration j gathers Vb_j's neighbours for Zb_j = Vb_j - lambda (2 gr Lr Vb_j
// + 2 gc Vb_j Lc), carries it to Sb_{j-1} = (1 + mu_{j-1}) Zb_j + A2 and
// A2 = -mu_{j-1} Zb_j, and forms and publishes Vb_{j-1} (dY~ += Sb - Vb)
// for the next iteration; the launch's last iteration leaves Sb_{j-1} in Sb
// instead (the next launch's prologue applies M_{j-1}, which the earlier
// segment's forward provides). The dL partial sums pair Vb_j with Z_j's
// neighbours. The scalar derivatives use the symmetry of Lr and Lc:
// <Vb, Lr Z> = <Lr Vb, Z> and <Vb, Z Lc> = <Vb Lc, Z>, so they come from the
// same gathers:
//   dgamma_r = -2 lambda <Lr Vb, Z>, dgamma_c = -2 lambda <Vb Lc, Z>,
//   dlambda = sum -sgn(V - Y~) Vb - (2 gr <Lr Vb, Z> + 2 gc <Vb Lc, Z>).
// RESIDENT: one tile per block for the whole launch (lists staged once, the
// staged entries' dL partial sums kept in shared memory in FP32 and added to
// the FP64 partial buffers at the end); otherwise blocks stream over tiles.
template <bool RESIDENT>
__global__ void __launch_bounds__(256, RESIDENT ? 5 : 4)
traj_reverse_kernel(const __grid_constant__ TrajArgs a) {
  using Off = typename std::conditional<RESIDENT, int32_t, int64_t>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  TrajSmem<Off>& sm = *reinterpret_cast<TrajSmem<Off>*>(smraw);
  __shared__ double red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = warp * 4 + (lane >> 3), cq = 4 * (lane & 7);
  const float lam = float(*a.lam);
  const double lamd = double(lam);
  const int64_t nnz_r = a.Lr.rowptr[a.rr], nnz_c = a.Lc.rowptr[a.rc];
  const double sr = -2.0 * lamd * a.gamma_r, sc = -2.0 * lamd * a.gamma_c;
  if (RESIDENT) {
    int i0, j0, ni, nj;
    tile_of(a, blockIdx.x, i0, j0, ni, nj);
    stage_nbr(sm.nb, a.Lr, a.Lc, int(a.ldzt), int(a.ldz), i0, j0, ni, nj);
    for (int e = threadIdx.x; e < TB * kTileNbr; e += blockDim.x) {
      sm.pr[e / kTileNbr][e % kTileNbr] = 0.f;
      sm.pc[e / kTileNbr][e % kTileNbr] = 0.f;
    }
  }
  double s_sgn = 0.0, s_r = 0.0, s_c = 0.0;  // sum -sgn Vb, <Lr Vb, Z>, <Vb Lc, Z>
  // transposed publish of the tile's new values through sm.tl
  auto publish_t = [&](const float4& v4, float* VT, int i0, int j0, int ni, int nj) {
    sm.tl[rl][cq] = v4.x;
    sm.tl[rl][cq + 1] = v4.y;
    sm.tl[rl][cq + 2] = v4.z;
    sm.tl[rl][cq + 3] = v4.w;
    __syncthreads();
    if (rl < nj && cq < ni)
      *reinterpret_cast<float4*>(VT + int64_t(j0 + rl) * a.ldzt + i0 + cq) =
          make_float4(sm.tl[cq][rl], sm.tl[cq + 1][rl], sm.tl[cq + 2][rl], sm.tl[cq + 3][rl]);
  };
  // apply a prox code word to 4 entries of Sb: Vb, dY~ += Sb - Vb, the sign sum
  auto apply_mask = [&](const float4& sb4, uint32_t code, float4& dy4, int nv) {
    float4 vb4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nv) {
        const uint32_t c = (code >> (8 * q)) & 3u;
        const float sb = cmp(sb4, q);
        const float vb = (c & 1u) ? sb : 0.f;
        cmp(dy4, q) += sb - vb;
        if (vb != 0.f) s_sgn += (c & 2u) ? double(vb) : -double(vb);
        cmp(vb4, q) = vb;
      }
    return vb4;
  };
  // prologue: Vb_jb = M_jb o Sb
  {
    const int par = a.jb & 1;
    const uint8_t* Mj = mslot(a, a.jb);
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      int i0, j0, ni, nj;
      tile_of(a, tile, i0, j0, ni, nj);
      float4 vb4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rl < ni && cq < nj) {
        const int64_t i = i0 + rl, jj = j0 + cq, l = i * a.ldz + jj;
        const int nv = nj - cq;
        const float4 sb4 = *reinterpret_cast<const float4*>(a.Sb + l);
        const uint32_t code = *reinterpret_cast<const uint32_t*>(Mj + l);
        float4 dy4 = ld4(a.dY + i * a.lddy + jj, a.dyvec, nv);
        vb4 = apply_mask(sb4, code, dy4, nv);
        st4(a.dY + i * a.lddy + jj, dy4, a.dyvec, nv);
        *reinterpret_cast<float4*>(a.Vb[par] + l) = vb4;
      }
      publish_t(vb4, a.VbT[par], i0, j0, ni, nj);
      __syncthreads();
    }
  }
  if (!grid_sync(a.bar)) return;
  for (int j = a.jb; j >= a.ja; --j) {
    const int par = j & 1;
    const float* V = a.Vb[par];
    const float* VT = a.VbT[par];
    const float* Zin = zslot(a, j);
    const float* ZTin = ztslot(a, j);
    const float mup = j >= 2 ? a.mu[j - 1] : 0.f;
    const bool form = j >= 2 && j > a.ja;  // Vb_{j-1} formed here
    const uint8_t* Mn = form ? mslot(a, j - 1) : nullptr;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      int i0, j0, ni, nj;
      tile_of(a, tile, i0, j0, ni, nj);
      const int ti = i0 / TB, tj = j0 / TB;
      if (RESIDENT) __syncthreads();  // sm.ac / sm.tl of the previous iteration are consumed
      else stage_nbr(sm.nb, a.Lr, a.Lc, int(a.ldzt), int(a.ldz), i0, j0, ni, nj);
      {
        const float4 o = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.coff[rl], sm.nb.cval[rl], sm.nb.cdeg[rl],
                                                           sm.nb.cf0[rl], rl < nj && cq < ni, VT, i0 + cq,
                                                           a.Lc, a.ldzt);
        sm.ac[cq][rl] = o.x;
        sm.ac[cq + 1][rl] = o.y;
        sm.ac[cq + 2][rl] = o.z;
        sm.ac[cq + 3][rl] = o.w;
      }
      const bool own = rl < ni && cq < nj;
      const float4 ar = nbr_sum_v4<Off, RESIDENT ? 4 : 8>(sm.nb.roff[rl], sm.nb.rval[rl], sm.nb.rdeg[rl],
                                                          sm.nb.rf0[rl], own, V, j0 + cq, a.Lr, a.ldz);
      __syncthreads();
      float4 vb4 = make_float4(0.f, 0.f, 0.f, 0.f), vn4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (own) {
        const int64_t i = i0 + rl, jj = j0 + cq, l = i * a.ldz + jj;
        const int nv = nj - cq;
        vb4 = __ldcg(reinterpret_cast<const float4*>(V + l));
        const float4 z4 = __ldcg(reinterpret_cast<const float4*>(Zin + l));
        const float4 a24 = *reinterpret_cast<const float4*>(a.A2 + l);
        float4 zb4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nv) {
            const float arq = cmp(ar, q), acq = sm.ac[rl][cq + q];
            cmp(zb4, q) = fmaf(-lam, fmaf(a.two_gr, arq, a.two_gc * acq), cmp(vb4, q));
            s_r += double(arq) * double(cmp(z4, q));
            s_c += double(acq) * double(cmp(z4, q));
          }
        if (j >= 2) {
          float4 sbn = make_float4(0.f, 0.f, 0.f, 0.f), a2n = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < nv) {
              cmp(sbn, q) = fmaf(1.f + mup, cmp(zb4, q), cmp(a24, q));
              cmp(a2n, q) = -mup * cmp(zb4, q);
            }
          *reinterpret_cast<float4*>(a.A2 + l) = a2n;
          if (form) {
            const uint32_t code = *reinterpret_cast<const uint32_t*>(Mn + l);
            float4 dy4 = ld4(a.dY + i * a.lddy + jj, a.dyvec, nv);
            vn4 = apply_mask(sbn, code, dy4, nv);
            st4(a.dY + i * a.lddy + jj, dy4, a.dyvec, nv);
            *reinterpret_cast<float4*>(a.Vb[par ^ 1] + l) = vn4;
          } else {
            *reinterpret_cast<float4*>(a.Sb + l) = sbn;
          }
        } else {
          float4 dy4 = ld4(a.dY + i * a.lddy + jj, a.dyvec, nv);
#pragma unroll
          for (int q = 0; q < 4; ++q) cmp(dy4, q) += cmp(zb4, q) + cmp(a24, q);
          st4(a.dY + i * a.lddy + jj, dy4, a.dyvec, nv);
          *reinterpret_cast<float4*>(a.Sb + l) = make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(a.A2 + l) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      // dLr(a, b) += scale sum_c Vb(a, c) Z(b, c) over the tile's columns;
      // dLc(a, b) += scale sum_r Z(r, a) Vb(r, b) over its rows (column b's
      // list (b, a) lands on the transposed entry (a, b))
      const bool ocol = rl < nj && cq < ni;
      const float4 vc4 = ocol ? __ldcg(reinterpret_cast<const float4*>(VT + int64_t(j0 + rl) * a.ldzt + i0 + cq))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.gamma_r != 0.0)
        list_partials<RESIDENT>(sm.nb.roff[rl], sm.nb.rdeg[rl], sm.nb.rf0[rl], own, Zin, j0 + cq, a.Lr, a.ldz,
                                vb4, sm.pr[rl], sr, a.Pr + int64_t(tj) * nnz_r, nullptr, lane);
      if (a.gamma_c != 0.0)
        list_partials<RESIDENT>(sm.nb.coff[rl], sm.nb.cdeg[rl], sm.nb.cf0[rl], ocol, ZTin, i0 + cq, a.Lc,
                                a.ldzt, vc4, sm.pc[rl], sc, a.Pc + int64_t(ti) * nnz_c, a.tmap_c, lane);
      if (form) publish_t(vn4, a.VbT[par ^ 1], i0, j0, ni, nj);
      if (!RESIDENT) __syncthreads();
    }
    if (!grid_sync(a.bar)) return;
  }
  if (RESIDENT) {
    __syncthreads();
    int i0, j0, ni, nj;
    tile_of(a, blockIdx.x, i0, j0, ni, nj);
    double* Prt = a.Pr + int64_t(j0 / TB) * nnz_r;
    double* Pct = a.Pc + int64_t(i0 / TB) * nnz_c;
    // flush the staged entries' partial sums: row lists on their own
    // entries of Lr, column lists on the transposed entries of Lc
    for (int e = threadIdx.x; e < TB * kTileNbr; e += blockDim.x) {
      const int r = e / kTileNbr, q = e % kTileNbr;
      const float vr = sm.pr[r][q];
      if (vr != 0.f) Prt[sm.nb.rf0[r] + q] += sr * double(vr);
      const float vc = sm.pc[r][q];
      if (vc != 0.f) {
        const int64_t t = __ldg(a.tmap_c + sm.nb.cf0[r] + q);
        if (t >= 0) Pct[t] += sc * double(vc);
      }
    }
  }
  s_sgn = block_sum(s_sgn, red);
  s_r = block_sum(s_r, red);
  s_c = block_sum(s_c, red);
  if (threadIdx.x == 0) {
    atomicAdd(a.scal_bar + 0, s_sgn - (2.0 * a.gamma_r * s_r + 2.0 * a.gamma_c * s_c));
    atomicAdd(a.scal_bar + 1, -2.0 * lamd * s_r);
    atomicAdd(a.scal_bar + 2, -2.0 * lamd * s_c);
  }
}

// dL(e) = sum over parts p of P[p][e], in order.
__global__ void reduce_parts_kernel(const double* __restrict__ P, int nparts, int64_t nnz,
                                    double* __restrict__ out) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz;
       e += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += P[int64_t(p) * nnz + e];
    out[e] = s;
  }
}

// ------------------------------------------------------ power iteration --
// The solve's power iteration, with every iterate kept: u_0(i) = uniform - 1/2
// (SplitMix64 stream 2 for Lr, 3 for Lc), u_{t+1} = (L u_t) / |u_t|, and
// rho = u_T^T L u_T / u_T^T u_T. Reverse mode with v_t = u_t / |u_t|:
//   vbar_T = 2 rhobar (L v_T - rho v_T), dL += rhobar v_T v_T^T;
//   t = T..1: ubar_t = (vbar_t - v_t (v_t^T vbar_t)) / |u_t|,
//             dL += ubar_t v_{t-1}^T, vbar_{t-1} = L ubar_t.
struct PowGraph {
  CsrView L;
  int n, stream, row0;
  float* U;       // [(T + 1) * n], iterate t at U + t * n
  double* nrm2;   // [T + 1]
  float* Ub;      // [T * n], ubar_t at Ub + (t - 1) * n
  float* vb[2];   // vbar ping-pong
  double* acc;    // [4]: ring of dot products
  double* fin;    // [2]: u^T L u, u^T u
  double* rho;    // out: estimate
  const double* rho_bar;
};
struct PowAdjArgs {
  PowGraph g[2];
  int rows, T;
  uint64_t seed;
  int reverse;
  GridBar bar;
};

__device__ __forceinline__ int pow_graph(const PowAdjArgs& a, int r) { return r >= a.g[1].row0 ? 1 : 0; }

__device__ __forceinline__ float spmv_row(const CsrView& L, int i, const float* x, float scale, int lane) {
  float sum = 0.f;
  for (int64_t e = L.rowptr[i] + lane; e < L.rowptr[i + 1]; e += 32)
    sum = fmaf(__ldg(L.val + e), __ldcg(x + __ldg(L.col + e)), sum);
  return warp_sumf(sum) * scale;
}

// Two per-graph FP64 sums, added up in the block first (shared atomics) and
// then with one global atomic per block and graph.
__device__ __forceinline__ void flush2(double* bs, double* g0, double* g1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bs[0] != 0.0) atomicAdd(g0, bs[0]);
    if (bs[1] != 0.0) atomicAdd(g1, bs[1]);
    bs[0] = bs[1] = 0.0;
  }
}

__global__ void __launch_bounds__(512)
power_adjoint_kernel(const __grid_constant__ PowAdjArgs a) {
  __shared__ double bs[2];
  if (threadIdx.x < 2) bs[threadIdx.x] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nthr = gridDim.x * blockDim.x, tid = blockIdx.x * blockDim.x + threadIdx.x;
  // each warp keeps its first row's CSR entries in registers (at most 32)
  int c_d = -1, c_col = 0;
  float c_val = 0.f;
  if (wid < a.rows) {
    const PowGraph& G = a.g[pow_graph(a, wid)];
    const int i = wid - G.row0;
    const int64_t e0 = G.L.rowptr[i];
    c_d = int(G.L.rowptr[i + 1] - e0);
    if (c_d <= 32 && lane < c_d) {
      c_col = G.L.col[e0 + lane];
      c_val = G.L.val[e0 + lane];
    }
  }
  // row r's product with x (scaled): from the registers when cached
  auto row_dot = [&](const PowGraph& G, int r, const float* x, float scale) -> float {
    if (r == wid && c_d >= 0 && c_d <= 32) return warp_sumf(lane < c_d ? c_val * __ldcg(x + c_col) : 0.f) * scale;
    return spmv_row(G.L, r - G.row0, x, scale, lane);
  };
  if (!a.reverse) {
    for (int r = tid; r < a.rows; r += nthr) {
      const PowGraph& G = a.g[pow_graph(a, r)];
      const int i = r - G.row0;
      const double x = uniform01_at(stream_state0(a.seed, G.stream), uint64_t(i) + 1) - 0.5;
      G.U[i] = float(x);
      atomicAdd(bs + pow_graph(a, r), x * x);
    }
    flush2(bs, a.g[0].nrm2, a.g[1].nrm2);
    if (!grid_sync(a.bar)) return;
    for (int t = 0; t < a.T; ++t) {
      for (int r = wid; r < a.rows; r += nwarp) {
        const PowGraph& G = a.g[pow_graph(a, r)];
        const int i = r - G.row0;
        const double n2 = __ldcg(G.nrm2 + t);
        const float inv = n2 > 0 ? float(1.0 / sqrt(n2)) : 0.f;
        const float s = row_dot(G, r, G.U + size_t(t) * G.n, inv);
        if (lane == 0) {
          G.U[size_t(t + 1) * G.n + i] = s;
          atomicAdd(bs + pow_graph(a, r), double(s) * double(s));
        }
      }
      flush2(bs, a.g[0].nrm2 + t + 1, a.g[1].nrm2 + t + 1);
      if (!grid_sync(a.bar)) return;
    }
    for (int r = wid; r < a.rows; r += nwarp) {
      const PowGraph& G = a.g[pow_graph(a, r)];
      const int i = r - G.row0;
      const float* u = G.U + size_t(a.T) * G.n;
      const float s = spmv_row(G.L, i, u, 1.f, lane);
      if (lane == 0) {
        const double ui = __ldcg(u + i);
        atomicAdd(G.fin, ui * double(s));
        atomicAdd(G.fin + 1, ui * ui);
      }
    }
    if (!grid_sync(a.bar)) return;
    if (blockIdx.x == 0 && threadIdx.x < 2) {
      const PowGraph& G = a.g[threadIdx.x];
      const double num = __ldcg(G.fin), den = __ldcg(G.fin + 1);
      *G.rho = (den > 0 && __ldcg(G.nrm2 + a.T) > 0) ? num / den : 0.0;
    }
    return;
  }
  // reverse: vbar_T = 2 rhobar (L v_T - rho v_T); dot v_T . vbar_T into acc[T % 4]
  for (int r = wid; r < a.rows; r += nwarp) {
    const PowGraph& G = a.g[pow_graph(a, r)];
    const int i = r - G.row0;
    const double n2 = __ldcg(G.nrm2 + a.T);
    const double inv = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
    const float* u = G.U + size_t(a.T) * G.n;
    const float lv = row_dot(G, r, u, 1.f);
    if (lane == 0) {
      const double vi = double(__ldcg(u + i)) * inv;
      const double vb = 2.0 * (*G.rho_bar) * (double(lv) * inv - (*G.rho) * vi);
      G.vb[a.T & 1][i] = float(vb);
      atomicAdd(bs + pow_graph(a, r), vi * vb);
    }
  }
  flush2(bs, a.g[0].acc + (a.T & 3), a.g[1].acc + (a.T & 3));
  if (!grid_sync(a.bar)) return;
  for (int t = a.T; t >= 1; --t) {
    // ubar_t = (vbar_t - v_t d_t) / |u_t|
    for (int r = tid; r < a.rows; r += nthr) {
      const PowGraph& G = a.g[pow_graph(a, r)];
      const int i = r - G.row0;
      const double n2 = __ldcg(G.nrm2 + t);
      const double inv = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
      const double d = __ldcg(G.acc + (t & 3));
      const double vi = double(G.U[size_t(t) * G.n + i]) * inv;
      G.Ub[size_t(t - 1) * G.n + i] = float((double(G.vb[t & 1][i]) - vi * d) * inv);
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) a.g[threadIdx.x].acc[(t + 2) & 3] = 0.0;
    if (!grid_sync(a.bar)) return;
    // vbar_{t-1} = L ubar_t; dot v_{t-1} . vbar_{t-1}
    for (int r = wid; r < a.rows; r += nwarp) {
      const PowGraph& G = a.g[pow_graph(a, r)];
      const int i = r - G.row0;
      const float s = row_dot(G, r, G.Ub + size_t(t - 1) * G.n, 1.f);
      if (lane == 0) {
        G.vb[(t - 1) & 1][i] = s;
        if (t > 1) {
          const double n2 = __ldcg(G.nrm2 + t - 1);
          const double inv = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
          atomicAdd(bs + pow_graph(a, r), double(G.U[size_t(t - 1) * G.n + i]) * inv * double(s));
        }
      }
    }
    flush2(bs, a.g[0].acc + ((t - 1) & 3), a.g[1].acc + ((t - 1) & 3));
    if (!grid_sync(a.bar)) return;
  }
}

// dL(e) += rhobar v_T(i) v_T(j) + sum_t ubar_t(i) v_{t-1}(j), e = (i, j).
__global__ void power_pattern_kernel(PowGraph G, int T, double* __restrict__ dL) {
  const double rb = *G.rho_bar;
  if (rb == 0.0) return;
  for (int i = blockIdx.x; i < G.n; i += gridDim.x)
    for (int64_t e = G.L.rowptr[i] + threadIdx.x; e < G.L.rowptr[i + 1]; e += blockDim.x) {
      const int j = G.L.col[e];
      const double nT = G.nrm2[T];
      double s = nT > 0 ? rb * double(G.U[size_t(T) * G.n + i]) * double(G.U[size_t(T) * G.n + j]) / nT : 0.0;
      for (int t = 1; t <= T; ++t) {
        const double n2 = G.nrm2[t - 1];
        if (n2 > 0)
          s += double(G.Ub[size_t(t - 1) * G.n + i]) * double(G.U[size_t(t - 1) * G.n + j]) / sqrt(n2);
      }
      dL[e] += s;
    }
}

// lambda = 1/beta', beta' = 2 gamma_c n_c + 2 gamma_r n_r: the solve's step
// and the chain rule back to gamma and the norm estimates.
// scal: [0] n_r, [1] n_c, [2] lambda; bar: [0] dlambda, [1] dgamma_r, [2] dgamma_c,
// out nb: [0] dn_r, [1] dn_c.
__global__ void step_forward_kernel(double* scal, double gr, double gc, double step) {
  if (threadIdx.x || blockIdx.x) return;
  if (step > 0) {
    scal[2] = step;
  } else {
    const double beta = 2.0 * gc * scal[1] + 2.0 * gr * scal[0];
    scal[2] = beta > 0 ? 1.0 / beta : 1.0;
  }
}
__global__ void step_backward_kernel(const double* scal, double* bar, double* nb, double gr, double gc,
                                     double step) {
  if (threadIdx.x || blockIdx.x) return;
  nb[0] = nb[1] = 0.0;
  if (step > 0) return;
  const double beta = 2.0 * gc * scal[1] + 2.0 * gr * scal[0];
  if (!(beta > 0)) return;
  const double d = -bar[0] / (beta * beta);
  bar[1] += 2.0 * scal[0] * d;
  bar[2] += 2.0 * scal[1] * d;
  nb[0] = 2.0 * gr * d;
  nb[1] = 2.0 * gc * d;
}

// ------------------------------------------------------ weight chain rule --
// The Laplacians of Sec. I as functions of the symmetric edge weights w:
//   normalised      L_ij = -w_ij / sqrt(D_i D_j) (i != j), L_ii = [D_i > 0];
//   combinatorial   L_ij = -w_ij, L_ii = D_i;   D_i = sum_j w_ij.
// Given dL on the pattern, the derivative of an undirected edge {i, j}:
//   normalised:     -(dL_ij + dL_ji) / sqrt(D_i D_j) + dD_i + dD_j,
//                   dD_k = -sum_{l != k} (dL_kl + dL_lk) L_kl / (2 D_k);
//   combinatorial:  -(dL_ij + dL_ji) + dL_ii + dL_jj;
// written at both entries ij and ji (0 on the diagonal).
__device__ __forceinline__ int64_t find_entry(const CsrView& L, int row, int col) {
  int64_t lo = L.rowptr[row], hi = L.rowptr[row + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (L.col[mid] < col) lo = mid + 1; else hi = mid;
  }
  return (lo < L.rowptr[row + 1] && L.col[lo] == col) ? lo : -1;
}

__global__ void transpose_map_kernel(CsrView L, int64_t* __restrict__ tmap) {
  for (int i = blockIdx.x; i < L.n; i += gridDim.x)
    for (int64_t e = L.rowptr[i] + threadIdx.x; e < L.rowptr[i + 1]; e += blockDim.x)
      tmap[e] = find_entry(L, L.col[e], i);
}

__global__ void wchain_node_kernel(CsrView L, const float* __restrict__ w, const double* __restrict__ dL,
                                   int lap_type, double* __restrict__ deg, double* __restrict__ dD) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
    double d = 0.0, s = 0.0, diag = 0.0;
    for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e) {
      const int j = L.col[e];
      if (j == i) {
        diag = dL[e];
        continue;
      }
      d += double(w[e]);
      const int64_t et = find_entry(L, j, i);
      s += (dL[e] + (et >= 0 ? dL[et] : 0.0)) * double(L.val[e]);
    }
    deg[i] = d;
    if (lap_type == 1) dD[i] = diag;
    else dD[i] = d > 0 ? -s / (2.0 * d) : 0.0;
  }
}

__global__ void wchain_edge_kernel(CsrView L, const double* __restrict__ dL, int lap_type,
                                   const double* __restrict__ deg, const double* __restrict__ dD,
                                   float* __restrict__ dw) {
  for (int i = blockIdx.x; i < L.n; i += gridDim.x)
    for (int64_t e = L.rowptr[i] + threadIdx.x; e < L.rowptr[i + 1]; e += blockDim.x) {
      const int j = L.col[e];
      if (j == i) {
        dw[e] = 0.f;
        continue;
      }
      const int64_t et = find_entry(L, j, i);
      const double both = dL[e] + (et >= 0 ? dL[et] : 0.0);
      double g;
      if (lap_type == 1) g = -both + dD[i] + dD[j];
      else g = -both / sqrt(deg[i] * deg[j]) + dD[i] + dD[j];
      dw[e] = float(g);
    }
}

// Laplacian values from the weights (Sec. I): D_i = sum_j w_ij in FP64;
// normalised: -w_ij / sqrt(D_i D_j) off the diagonal, [D_i > 0] on it;
// combinatorial: -w_ij, D_i.
__global__ void degree_kernel(CsrView L, const float* __restrict__ w, double* __restrict__ deg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e)
      if (L.col[e] != i) d += double(w[e]);
    deg[i] = d;
  }
}
__global__ void lap_values_kernel(CsrView L, const float* __restrict__ w, const double* __restrict__ deg,
                                  int lap_type, float* __restrict__ val) {
  for (int i = blockIdx.x; i < L.n; i += gridDim.x)
    for (int64_t e = L.rowptr[i] + threadIdx.x; e < L.rowptr[i + 1]; e += blockDim.x) {
      const int j = L.col[e];
      double v;
      if (lap_type == 1) v = j == i ? deg[i] : -double(w[e]);
      else if (j == i) v = deg[i] > 0 ? 1.0 : 0.0;
      else v = (deg[i] > 0 && deg[j] > 0) ? -double(w[e]) / sqrt(deg[i] * deg[j]) : 0.0;
      val[e] = float(v);
    }
}

struct BwdWs {
  float* mu;
  double* scal;      // [4]: n_r, n_c, lambda
  double* bar;       // [4]: dlambda, dgamma_r, dgamma_c
  double* nb;        // [2]: dn_r, dn_c
  float *S, *Sb, *A2, *Vb[2], *VbT[2];
  float *Zs, *ZTs;
  uint8_t* Ms;
  void* pscr;        // power iteration scratch (grid-wide kernel)
  float *ckS, *ckZ;
  double *Pr, *Pc;
  double *dLr, *dLc;
  double *deg, *dD;
  int64_t* tmap_c;
  float* U[2];
  double* nrm2[2];
  float* Ub[2];
  float* vb[2][2];
  double* pacc;      // [2][4] + fin [2][2] + rho [2]
  unsigned int* bar_cnt;
  int* err;
  size_t bytes;
};

BwdWs bwd_layout(void* ws, int rr, int rc, int J, int ck, int T, int64_t nnz_r, int64_t nnz_c) {
  Carve c(ws);
  BwdWs w{};
  // row-major buffers rr x ldz, column-major rc x ldzt (rows padded to 4)
  const size_t mn = size_t(rr) * ((rc + 3) / 4 * 4), mnt = size_t(rc) * ((rr + 3) / 4 * 4);
  const int nseg = (J + ck - 1) / ck;
  const int nslot = std::max(ck + 1, 2);
  w.mu = c.take<float>(size_t(J) + 2);
  w.scal = c.take<double>(4);
  w.bar = c.take<double>(4);
  w.nb = c.take<double>(2);
  w.S = c.take<float>(mn);
  w.Sb = c.take<float>(mn);
  w.A2 = c.take<float>(mn);
  for (int p = 0; p < 2; ++p) {
    w.Vb[p] = c.take<float>(mn);
    w.VbT[p] = c.take<float>(mnt);
  }
  w.Zs = c.take<float>(mn * nslot);
  w.ZTs = c.take<float>(mnt * nslot);
  w.Ms = c.take<uint8_t>(mn * nslot);
  w.ckS = c.take<float>(mn * std::max(nseg - 1, 1));
  w.ckZ = c.take<float>(mn * std::max(nseg - 1, 1));
  w.Pr = c.take<double>(size_t(ceil_div(rc, TB)) * std::max<int64_t>(nnz_r, 1));
  w.Pc = c.take<double>(size_t(ceil_div(rr, TB)) * std::max<int64_t>(nnz_c, 1));
  w.dLr = c.take<double>(std::max<int64_t>(nnz_r, 1));
  w.dLc = c.take<double>(std::max<int64_t>(nnz_c, 1));
  w.deg = c.take<double>(std::max(rr, rc));
  w.dD = c.take<double>(std::max(rr, rc));
  w.tmap_c = c.take<int64_t>(std::max<int64_t>(nnz_c, 1));
  for (int g = 0; g < 2; ++g) {
    const int n = g ? rc : rr;
    w.U[g] = c.take<float>(size_t(T + 1) * n);
    w.nrm2[g] = c.take<double>(size_t(T) + 1);
    w.Ub[g] = c.take<float>(size_t(std::max(T, 1)) * n);
    w.vb[g][0] = c.take<float>(n);
    w.vb[g][1] = c.take<float>(n);
  }
  w.pacc = c.take<double>(16);
  {
    const int ns[2] = {rr, rc};
    w.pscr = c.take<unsigned char>(power_scratch_bytes(ns, 2));
  }
  w.bar_cnt = c.take<unsigned int>(kBarrierCounters + 1);
  w.err = c.take<int>(1);
  w.bytes = c.bytes();
  return w;
}

cpca_status reset_barrier(const BwdWs& w, cudaStream_t st) {
  CPCA_CUDA(cudaMemsetAsync(w.bar_cnt, 0, sizeof(unsigned int) * (kBarrierCounters + 1), st));
  return CPCA_OK;
}

cpca_status run_power(PowAdjArgs& pa, const BwdWs& w, int reverse, cudaStream_t st) {
  const CsrView Ls[2] = {pa.g[0].L, pa.g[1].L};
  if (!reverse || power_tape_fits(Ls, 2)) {  // the solve's power kernels (reverse: one cluster)
    PowerTape P[2];
    for (int g = 0; g < 2; ++g) {
      const PowGraph& G = pa.g[g];
      P[g] = PowerTape{G.L, G.stream, G.U, G.nrm2, G.Ub, G.rho, G.rho_bar};
    }
    CPCA_PROF(reverse ? "adj_power_rev" : "adj_power_fwd", st);
    return power_tape_run(P, 2, pa.T, pa.seed, reverse != 0, w.pscr, w.bar_cnt, w.err, st);
  }
  pa.reverse = reverse;
  CPCA_TRY(reset_barrier(w, st));
  const int want = ceil_div(int64_t(pa.rows) * 32, 512);
  const int grid = std::min(2 * num_sms(), coop_blocks((const void*)power_adjoint_kernel, 512, 0,
                                                       std::max(want, 1)));
  void* args[] = {&pa};
  CPCA_PROF(reverse ? "adj_power_rev" : "adj_power_fwd", st);
  CPCA_CUDA(cudaLaunchCooperativeKernel((void*)power_adjoint_kernel, dim3(grid), dim3(512), args, 0, st));
  CPCA_LAUNCHED();
  return CPCA_OK;
}

cpca_status weight_chain(const CsrView& L, const float* w, const double* dL, int lap_type, float* dw,
                         const BwdWs& ws, cudaStream_t st) {
  const unsigned g = std::min<unsigned>(ceil_div(L.n, 256), num_sms() * 4);
  wchain_node_kernel<<<g, 256, 0, st>>>(L, w, dL, lap_type, ws.deg, ws.dD);
  CPCA_LAUNCHED();
  wchain_edge_kernel<<<std::min(L.n, num_sms() * 8), 64, 0, st>>>(L, dL, lap_type, ws.deg, ws.dD, dw);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

}  // namespace

// Chain rule from dL (FP64, on the CSR pattern) to the edge weights; shared
// with the decoder's derivative.
cpca_status laplacian_weight_grad(const CsrView& L, const float* w, const double* dL, int lap_type,
                                  float* dw, double* deg, double* dD, cudaStream_t st) {
  BwdWs ws{};
  ws.deg = deg;
  ws.dD = dD;
  return weight_chain(L, w, dL, lap_type, dw, ws, st);
}

}  // namespace cpca

using namespace cpca;

extern "C" size_t cpca_frpcag_backward_workspace_size(int32_t rr, int32_t rc, int32_t max_iter,
                                                      int32_t ckpt_every, int32_t power_iters,
                                                      int64_t nnz_r, int64_t nnz_c) {
  if (rr <= 0 || rc <= 0 || max_iter < 1 || ckpt_every < 0 || power_iters < 0 || nnz_r < 0 || nnz_c < 0)
    return 0;
  const int ck = std::min(ckpt_every > 0 ? ckpt_every : 20, int(max_iter));
  return bwd_layout(nullptr, rr, rc, max_iter, ck, power_iters, nnz_r, nnz_c).bytes;
}

namespace {

enum AdjMode { kForwardTape, kBackward, kBackwardResume };

struct AdjCall {
  const float* Yt;
  int rr, rc;
  int64_t ldyt;
  const cpca_csr *Lr, *Lc;
  const cpca_frpcag_params* prm;
  int ckpt_every;
  // forward tape: X out
  float* X;
  int64_t ldx;
  // backward
  const float* dX;
  int64_t lddx;
  float* dYt;
  int64_t lddyt;
  double *dLr, *dLc;
  const float *wr, *wc;
  int lap_type;
  float *dwr, *dwc;
  cpca_frpcag_grad_info* ginfo;
  void* ws;
  size_t ws_bytes;
  cudaStream_t st;
};

cpca_status check_adj(const AdjCall& c, const char* who) {
  CPCA_CHECK_ARG(c.Yt && c.prm, "%s: null pointer", who);
  CPCA_CHECK_ARG(c.rr > 0 && c.rc > 0, "%s: empty matrix", who);
  CPCA_CHECK_ARG(c.ldyt >= c.rc, "%s: ldyt < rc", who);
  CPCA_CHECK_ARG(c.prm->max_iter >= 1, "%s: max_iter < 1", who);
  CPCA_CHECK_ARG(c.prm->eps == 0.0, "%s: needs a fixed iteration count (eps = 0)", who);
  CPCA_CHECK_ARG(c.prm->gamma_r >= 0 && c.prm->gamma_c >= 0, "%s: negative gamma", who);
  CPCA_CHECK_ARG(c.prm->step > 0 || c.prm->power_iters >= 1, "%s: power_iters < 1", who);
  CPCA_CHECK_ARG(c.ckpt_every >= 0, "%s: ckpt_every < 0", who);
  CPCA_CHECK_ARG(c.prm->start_iter == 0 && !c.prm->prev_out,
                 "%s: differentiates a cold-started solve (start_iter = 0, no prev_out)", who);
  CPCA_TRY(check_csr(c.Lr, c.rr, who));
  CPCA_TRY(check_csr(c.Lc, c.rc, who));
  return CPCA_OK;
}

// The forward tape (power iterates, lambda, momentum table, checkpoints)
// and the reverse sweeps, sharing one workspace layout.
cpca_status frpcag_adjoint(const AdjCall& c, AdjMode mode) {
  const int rr = c.rr, rc = c.rc;
  const cpca_frpcag_params* prm = c.prm;
  const int J = prm->max_iter;
  const int ck = std::min(c.ckpt_every > 0 ? c.ckpt_every : 20, J);
  const int T = prm->step > 0 ? 0 : prm->power_iters;
  const BwdWs w = bwd_layout(c.ws, rr, rc, J, ck, T, c.Lr->nnz, c.Lc->nnz);
  if (!c.ws || c.ws_bytes < w.bytes) {
    set_error("cpca_frpcag_backward: workspace %zu bytes < required %zu", c.ws_bytes, w.bytes);
    return CPCA_ERR_WORKSPACE;
  }
  cudaStream_t st = c.st;
  const CsrView lr{c.Lr->n, c.Lr->rowptr, c.Lr->col, c.Lr->val};
  const CsrView lc{c.Lc->n, c.Lc->rowptr, c.Lc->col, c.Lc->val};
  const int64_t ldz = (rc + 3) / 4 * 4, ldzt = (rr + 3) / 4 * 4;
  const size_t mn = size_t(rr) * ldz;
  CPCA_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));

  PowAdjArgs pa{};
  pa.rows = rr + rc;
  pa.T = T;
  pa.seed = prm->power_seed;
  pa.bar = grid_bar(w.bar_cnt, w.err);
  for (int g = 0; g < 2; ++g) {
    PowGraph& G = pa.g[g];
    G.L = g ? lc : lr;
    G.n = g ? rc : rr;
    G.stream = g ? 3 : 2;
    G.row0 = g ? rr : 0;
    G.U = w.U[g];
    G.nrm2 = w.nrm2[g];
    G.Ub = w.Ub[g];
    G.vb[0] = w.vb[g][0];
    G.vb[1] = w.vb[g][1];
    G.acc = w.pacc + 4 * g;
    G.fin = w.pacc + 8 + 2 * g;
    G.rho = w.scal + g;
    G.rho_bar = w.nb + g;
  }
  if (mode != kBackwardResume) {
    // power iterations with the iterates kept, then lambda and mu_j
    CPCA_CUDA(cudaMemsetAsync(w.scal, 0, 4 * sizeof(double), st));
    CPCA_CUDA(cudaMemsetAsync(w.pacc, 0, 16 * sizeof(double), st));
    if (T > 0) {
      for (int g = 0; g < 2; ++g) CPCA_CUDA(cudaMemsetAsync(w.nrm2[g], 0, sizeof(double) * (T + 1), st));
      CPCA_TRY(run_power(pa, w, 0, st));
    }
    step_forward_kernel<<<1, 32, 0, st>>>(w.scal, prm->gamma_r, prm->gamma_c, prm->step);
    CPCA_LAUNCHED();
    mu_kernel<<<1, 32, 0, st>>>(J, w.mu);
    CPCA_LAUNCHED();
  }

  TrajArgs a{};
  a.Yt = c.Yt;
  a.ldy = c.ldyt;
  a.rr = rr;
  a.rc = rc;
  a.ntj = ceil_div(rc, TB);
  a.ntiles = int(ceil_div(rr, TB) * int64_t(a.ntj));
  a.ldz = ldz;
  a.ldzt = ldzt;
  a.yvec = c.ldyt % 4 == 0 && reinterpret_cast<uintptr_t>(c.Yt) % 16 == 0;
  a.dyvec = c.dYt && c.lddyt % 4 == 0 && reinterpret_cast<uintptr_t>(c.dYt) % 16 == 0;
  a.Lr = lr;
  a.Lc = lc;
  a.lam = w.scal + 2;
  a.two_gr = float(2.0 * prm->gamma_r);
  a.two_gc = float(2.0 * prm->gamma_c);
  a.gamma_r = prm->gamma_r;
  a.gamma_c = prm->gamma_c;
  a.mu = w.mu;
  a.S = w.S;
  a.Zs = w.Zs;
  a.ZTs = w.ZTs;
  a.Ms = nullptr;
  a.J = J;
  a.ckS = w.ckS;
  a.ckZ = w.ckZ;
  a.Sb = w.Sb;
  a.A2 = w.A2;
  for (int p = 0; p < 2; ++p) {
    a.Vb[p] = w.Vb[p];
    a.VbT[p] = w.VbT[p];
  }
  a.dY = c.dYt;
  a.lddy = c.lddyt;
  a.Pr = w.Pr;
  a.Pc = w.Pc;
  a.scal_bar = w.bar;
  a.tmap_c = w.tmap_c;
  a.bar = grid_bar(w.bar_cnt, w.err);
  const size_t smem = sizeof(TrajSmem<int64_t>);
  const size_t smem_res = sizeof(TrajSmem<int32_t>);
  static PerDeviceOnce attr;
  CPCA_CUDA(once_per_device(attr, [&] {
    cudaError_t e = cudaFuncSetAttribute((const void*)traj_forward_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)traj_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(smem_res));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)traj_reverse_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)traj_reverse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(smem_res));
    return e;
  }));
  const int gf = coop_blocks((const void*)traj_forward_kernel<false>, 256, smem, a.ntiles);
  const int gb = coop_blocks((const void*)traj_reverse_kernel<false>, 256, smem, a.ntiles);
  const bool resident = mn < (size_t(1) << 31) && size_t(rc) * ldzt < (size_t(1) << 31) &&
      coop_blocks((const void*)traj_reverse_kernel<true>, 256, smem_res, 1 << 30) >= a.ntiles;
  const bool resident_f = mn < (size_t(1) << 31) && size_t(rc) * ldzt < (size_t(1) << 31) &&
      coop_blocks((const void*)traj_forward_kernel<true>, 256, smem_res, 1 << 30) >= a.ntiles;
  auto launch_fwd = [&]() -> cpca_status {
    CPCA_TRY(reset_barrier(w, st));
    void* args[] = {&a};
    CPCA_PROF("adj_fista_fwd", st);
    if (resident_f)
      CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)traj_forward_kernel<true>, dim3(a.ntiles), dim3(256),
                                            args, smem_res, st));
    else
      CPCA_CUDA(cudaLaunchCooperativeKernel((const void*)traj_forward_kernel<false>, dim3(gf), dim3(256), args,
                                            smem, st));
    CPCA_LAUNCHED();
    return CPCA_OK;
  };
  const int nseg = (J + ck - 1) / ck;
  const unsigned gs = std::min<unsigned>(a.ntiles, num_sms() * 8);
  auto launch = [&](const void* k, int grid, size_t sm, const char* name) -> cpca_status {
    CPCA_TRY(reset_barrier(w, st));
    void* args[] = {&a};
    CPCA_PROF(name, st);
    CPCA_CUDA(cudaLaunchCooperativeKernel(k, dim3(grid), dim3(256), args, sm, st));
    CPCA_LAUNCHED();
    return CPCA_OK;
  };

  const int jlast = (nseg - 1) * ck;  // start of the last segment
  if (mode == kForwardTape) {
    // iterations 1..jlast with checkpoints at j = ck, 2 ck, ..., jlast;
    // then the last segment with its Z_j kept in the slots (the reverse
    // sweep starts there without recomputing it); X = S_J
    seed_kernel<<<gs, 256, 0, st>>>(c.Yt, c.ldyt, c.Yt, c.ldyt, rr, rc, ldz, ldzt, w.Zs, w.ZTs, w.S);
    CPCA_LAUNCHED();
    if (nseg > 1) {
      a.jbase = 1;
      a.nslot = 2;
      a.ja = 1;
      a.jb = jlast;
      a.ck = ck;
      a.Ms = nullptr;
      CPCA_TRY(launch_fwd());
      const size_t off = size_t(nseg - 2) * mn;
      seed_kernel<<<gs, 256, 0, st>>>(w.ckZ + off, ldz, w.ckS + off, ldz, rr, rc, ldz, ldzt, w.Zs, w.ZTs, w.S);
      CPCA_LAUNCHED();
    }
    a.jbase = jlast + 1;
    a.nslot = ck + 1;
    a.ja = jlast + 1;
    a.jb = J;
    a.ck = 0;
    a.Ms = w.Ms;  // prox codes of the last segment, for a resumed reverse
    CPCA_TRY(launch_fwd());
    CPCA_CUDA(cudaMemcpy2DAsync(c.X, sizeof(float) * c.ldx, w.S, sizeof(float) * ldz, sizeof(float) * rc, rr,
                                cudaMemcpyDeviceToDevice, st));
  } else if (mode == kBackward && nseg > 1) {
    // forward pass with checkpoints at j = ck, 2 ck, ..., (nseg - 1) ck
    seed_kernel<<<gs, 256, 0, st>>>(c.Yt, c.ldyt, c.Yt, c.ldyt, rr, rc, ldz, ldzt, w.Zs, w.ZTs, w.S);
    CPCA_LAUNCHED();
    a.jbase = 1;
    a.nslot = 2;
    a.ja = 1;
    a.jb = (nseg - 1) * ck;
    a.ck = ck;
    a.Ms = nullptr;
    CPCA_TRY(launch_fwd());
  }
  if (mode != kForwardTape) {
    // reverse, segment by segment
    CPCA_CUDA(cudaMemsetAsync(w.bar, 0, 4 * sizeof(double), st));
    transpose_map_kernel<<<std::max(1, std::min(rc, num_sms() * 8)), 64, 0, st>>>(lc, w.tmap_c);
    CPCA_LAUNCHED();
    CPCA_CUDA(cudaMemsetAsync(w.Sb, 0, sizeof(float) * mn, st));
    CPCA_CUDA(cudaMemcpy2DAsync(w.Sb, sizeof(float) * ldz, c.dX, sizeof(float) * c.lddx, sizeof(float) * rc,
                                rr, cudaMemcpyDeviceToDevice, st));
    CPCA_CUDA(cudaMemsetAsync(w.A2, 0, sizeof(float) * mn, st));
    CPCA_CUDA(cudaMemset2DAsync(c.dYt, sizeof(float) * c.lddyt, 0, sizeof(float) * rc, rr, st));
    CPCA_CUDA(cudaMemsetAsync(w.Pr, 0, sizeof(double) * a.ntj * std::max<int64_t>(c.Lr->nnz, 1), st));
    CPCA_CUDA(cudaMemsetAsync(w.Pc, 0, sizeof(double) * ceil_div(rr, TB) * std::max<int64_t>(c.Lc->nnz, 1), st));
    a.Ms = w.Ms;  // every reverse launch reads the prox codes of its segment
    for (int m = nseg - 1; m >= 0; --m) {
      const int j0 = m * ck, j1 = std::min(J, j0 + ck);
      a.jbase = j0 + 1;
      a.nslot = ck + 1;
      a.ck = 0;
      // the tape already holds the last segment's trajectory
      const bool have = mode == kBackwardResume && m == nseg - 1;
      if (!have) {
        if (m == 0) {
          seed_kernel<<<gs, 256, 0, st>>>(c.Yt, c.ldyt, c.Yt, c.ldyt, rr, rc, ldz, ldzt, w.Zs, w.ZTs, w.S);
        } else {
          const size_t off = size_t(m - 1) * mn;
          seed_kernel<<<gs, 256, 0, st>>>(w.ckZ + off, ldz, w.ckS + off, ldz, rr, rc, ldz, ldzt, w.Zs, w.ZTs,
                                          w.S);
        }
        CPCA_LAUNCHED();
      }
      if (!have) {
        // iterations j0 + 1..j1 again: Z_j and the prox codes of each
        a.ja = j0 + 1;
        a.jb = j1;
        CPCA_TRY(launch_fwd());
      }
      a.ja = j0 + 1;
      a.jb = j1;
      if (resident) CPCA_TRY(launch((const void*)traj_reverse_kernel<true>, a.ntiles, smem_res, "adj_fista_rev"));
      else CPCA_TRY(launch((const void*)traj_reverse_kernel<false>, gb, smem, "adj_fista_rev"));
    }
    double* oLr = c.dLr ? c.dLr : w.dLr;
    double* oLc = c.dLc ? c.dLc : w.dLc;
    if (c.Lr->nnz > 0) {
      reduce_parts_kernel<<<std::min<unsigned>(ceil_div(c.Lr->nnz, 256), num_sms() * 4), 256, 0, st>>>(
          w.Pr, a.ntj, c.Lr->nnz, oLr);
      CPCA_LAUNCHED();
    }
    if (c.Lc->nnz > 0) {
      reduce_parts_kernel<<<std::min<unsigned>(ceil_div(c.Lc->nnz, 256), num_sms() * 4), 256, 0, st>>>(
          w.Pc, int(ceil_div(rr, TB)), c.Lc->nnz, oLc);
      CPCA_LAUNCHED();
    }
    // lambda -> gamma and the norm estimates -> power iterations
    step_backward_kernel<<<1, 32, 0, st>>>(w.scal, w.bar, w.nb, prm->gamma_r, prm->gamma_c, prm->step);
    CPCA_LAUNCHED();
    if (T > 0) {
      CPCA_CUDA(cudaMemsetAsync(w.pacc, 0, 8 * sizeof(double), st));
      CPCA_TRY(run_power(pa, w, 1, st));
      for (int g = 0; g < 2; ++g) {
        const PowGraph& G = pa.g[g];
        power_pattern_kernel<<<std::min(G.n, num_sms() * 8), 64, 0, st>>>(G, T, g ? oLc : oLr);
        CPCA_LAUNCHED();
      }
    }
    if (c.dwr) CPCA_TRY(weight_chain(lr, c.wr, oLr, c.lap_type, c.dwr, w, st));
    if (c.dwc) CPCA_TRY(weight_chain(lc, c.wc, oLc, c.lap_type, c.dwc, w, st));
  }
  double hs[4], hb[4], hn[2];
  int err = 0;
  CPCA_CUDA(cudaMemcpyAsync(hs, w.scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(hb, w.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(hn, w.nb, sizeof(hn), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPCA_CUDA(cudaStreamSynchronize(st));
  if (err) {
    set_error("cpca_frpcag_backward: grid barrier timed out");
    return CPCA_ERR_TIMEOUT;
  }
  if (c.ginfo) {
    const bool bwd = mode != kForwardTape;
    c.ginfo->dgamma_r = bwd ? hb[1] : 0.0;
    c.ginfo->dgamma_c = bwd ? hb[2] : 0.0;
    c.ginfo->dlambda = bwd ? hb[0] : 0.0;
    c.ginfo->dnorm_r = bwd ? hn[0] : 0.0;
    c.ginfo->dnorm_c = bwd ? hn[1] : 0.0;
    c.ginfo->lambda = hs[2];
    c.ginfo->norm_r = hs[0];
    c.ginfo->norm_c = hs[1];
  }
  return CPCA_OK;
}

}  // namespace

extern "C" cpca_status cpca_frpcag_forward_tape(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                                const cpca_csr* Lr, const cpca_csr* Lc,
                                                const cpca_frpcag_params* prm, int32_t ckpt_every, float* X,
                                                int64_t ldx, cpca_frpcag_grad_info* ginfo, void* ws,
                                                size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_RANGE("cpca_frpcag_forward_tape");
  AdjCall c{};
  c.Yt = Yt;
  c.rr = rr;
  c.rc = rc;
  c.ldyt = ldyt;
  c.Lr = Lr;
  c.Lc = Lc;
  c.prm = prm;
  c.ckpt_every = ckpt_every;
  c.X = X;
  c.ldx = ldx;
  c.ginfo = ginfo;
  c.ws = ws;
  c.ws_bytes = ws_bytes;
  c.st = static_cast<cudaStream_t>(stream);
  CPCA_TRY(check_adj(c, "cpca_frpcag_forward_tape"));
  CPCA_CHECK_ARG(X && ldx >= rc, "cpca_frpcag_forward_tape: need X with ldx >= rc");
  return frpcag_adjoint(c, kForwardTape);
}

extern "C" cpca_status cpca_frpcag_backward(const float* Yt, int32_t rr, int32_t rc, int64_t ldyt,
                                            const cpca_csr* Lr, const cpca_csr* Lc,
                                            const cpca_frpcag_params* prm, int32_t ckpt_every, int32_t resume,
                                            const float* dX, int64_t lddx, float* dYt, int64_t lddyt,
                                            double* dLr, double* dLc, const float* wr, const float* wc,
                                            int32_t lap_type, float* dwr, float* dwc,
                                            cpca_frpcag_grad_info* ginfo, void* ws, size_t ws_bytes,
                                            void* stream) {
  clear_error();
  CPCA_RANGE("cpca_frpcag_backward");
  AdjCall c{};
  c.Yt = Yt;
  c.rr = rr;
  c.rc = rc;
  c.ldyt = ldyt;
  c.Lr = Lr;
  c.Lc = Lc;
  c.prm = prm;
  c.ckpt_every = ckpt_every;
  c.dX = dX;
  c.lddx = lddx;
  c.dYt = dYt;
  c.lddyt = lddyt;
  c.dLr = dLr;
  c.dLc = dLc;
  c.wr = wr;
  c.wc = wc;
  c.lap_type = lap_type;
  c.dwr = dwr;
  c.dwc = dwc;
  c.ginfo = ginfo;
  c.ws = ws;
  c.ws_bytes = ws_bytes;
  c.st = static_cast<cudaStream_t>(stream);
  CPCA_TRY(check_adj(c, "cpca_frpcag_backward"));
  CPCA_CHECK_ARG(dX && dYt, "cpca_frpcag_backward: null dX / dYt");
  CPCA_CHECK_ARG(lddx >= rc && lddyt >= rc, "cpca_frpcag_backward: leading dimension < rc");
  CPCA_CHECK_ARG(lap_type == CPCA_LAP_NORMALIZED || lap_type == CPCA_LAP_COMBINATORIAL,
                 "cpca_frpcag_backward: unknown lap_type");
  CPCA_CHECK_ARG(!dwr || wr, "cpca_frpcag_backward: dwr needs the weights wr");
  CPCA_CHECK_ARG(!dwc || wc, "cpca_frpcag_backward: dwc needs the weights wc");
  return frpcag_adjoint(c, resume ? kBackwardResume : kBackward);
}

static cpca_status check_pattern(const cpca_csr* L, const char* who) {
  CPCA_CHECK_ARG(L && L->rowptr && L->n >= 0 && L->nnz >= 0 && (L->nnz == 0 || L->col),
                 "%s: bad CSR pattern", who);
  return CPCA_OK;
}

extern "C" size_t cpca_laplacian_workspace_size(int32_t n) {
  return n < 0 ? 0 : 2 * sizeof(double) * size_t(std::max(n, 1)) + 256;
}

extern "C" cpca_status cpca_laplacian_values(const cpca_csr* pattern, const float* w, int32_t lap_type,
                                             float* val, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  CPCA_TRY(check_pattern(pattern, "cpca_laplacian_values"));
  CPCA_CHECK_ARG(w && val, "cpca_laplacian_values: null pointer");
  CPCA_CHECK_ARG(lap_type == CPCA_LAP_NORMALIZED || lap_type == CPCA_LAP_COMBINATORIAL,
                 "cpca_laplacian_values: unknown lap_type");
  if (!ws || ws_bytes < cpca_laplacian_workspace_size(pattern->n)) {
    set_error("cpca_laplacian_values: workspace too small");
    return CPCA_ERR_WORKSPACE;
  }
  if (pattern->n == 0) return CPCA_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const CsrView L{pattern->n, pattern->rowptr, pattern->col, nullptr};
  double* deg = static_cast<double*>(ws);
  degree_kernel<<<std::min<unsigned>(ceil_div(L.n, 256), num_sms() * 4), 256, 0, st>>>(L, w, deg);
  CPCA_LAUNCHED();
  lap_values_kernel<<<std::min(L.n, num_sms() * 8), 64, 0, st>>>(L, w, deg, lap_type, val);
  CPCA_LAUNCHED();
  return CPCA_OK;
}

extern "C" cpca_status cpca_laplacian_weight_grad(const cpca_csr* L, const float* w, const double* dL,
                                                  int32_t lap_type, float* dw, void* ws, size_t ws_bytes,
                                                  void* stream) {
  clear_error();
  CPCA_TRY(check_pattern(L, "cpca_laplacian_weight_grad"));
  CPCA_CHECK_ARG(w && dL && dw && (L->nnz == 0 || L->val), "cpca_laplacian_weight_grad: null pointer");
  CPCA_CHECK_ARG(lap_type == CPCA_LAP_NORMALIZED || lap_type == CPCA_LAP_COMBINATORIAL,
                 "cpca_laplacian_weight_grad: unknown lap_type");
  if (!ws || ws_bytes < cpca_laplacian_workspace_size(L->n)) {
    set_error("cpca_laplacian_weight_grad: workspace too small");
    return CPCA_ERR_WORKSPACE;
  }
  if (L->n == 0) return CPCA_OK;
  const CsrView lv{L->n, L->rowptr, L->col, L->val};
  double* deg = static_cast<double*>(ws);
  return laplacian_weight_grad(lv, w, dL, lap_type, dw, deg, deg + std::max(L->n, 1),
                               static_cast<cudaStream_t>(stream));
}
