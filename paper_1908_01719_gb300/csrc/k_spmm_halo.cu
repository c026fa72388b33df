// Halo-staged Krylov apply: the SpMM of one Jacobi COCG/CG iteration with the
// search-direction update and the deferred solution update fused in.
//
// Rows are grouped into tiles along a Morton curve of their node coordinates
// (HaloTiles, built on the host).  A block takes one tile and one slice of
// 32*NB right-hand sides (NB <= 2 columns per lane; a wider vector layout is
// split over blockIdx.y):
//   1. stage: for every halo row j of the tile (the union of the tile rows'
//      columns) copy z_j and, where needed, p_prev_j of the slice into shared
//      memory with asynchronous copies (cp.async: no register round trip, all
//      of a tile's copies in flight at once), then form p_j = z_j + beta p_prev_j
//      in place;
//   2. apply: for every owned row, q_i = sum_j L_ij p_j from shared memory
//      (L_ij = a A0_ij + bq2 q_r^2 MD_ij + i cq q_r (qhat . Pd)_ij, the step
//      operator of Appendix B / Appendix A built on the fly), the partial
//      inner product <p, q>, the store of p_i and the x update
//      x_i += alpha_prev p_prev_i that the previous iteration left pending
//      (its load is issued before the row's sums, so its latency is hidden);
//   3. the last block forms alpha = rho / <p, q>, marks the x update of every
//      active system pending and flips the p-buffer parity.
// On the Kuhn stencil a tile of ~20 rows has ~100 halo rows, so each X row is
// read ~5 times from L2 instead of ~15 times (one gather per nonzero), and all
// halo loads of a tile are independent, which hides their latency.  The
// search-direction and solution updates ride on the same loads, so the
// separate p-update kernel and the x part of the vector update disappear.
#include "bt_kernels.cuh"

namespace bt {

// columns per lane one block handles for a vector layout of nb columns per lane
__host__ __device__ constexpr int halo_nb(int nb) { return nb < 2 ? nb : 2; }
// staged entries of one tile: planes (float4), MD (float), local indices (uint16 in 4-byte words)
constexpr size_t HALO_ENTRY_BYTES = (size_t)HALO_EMAX * 16 + (size_t)HALO_EMAX * 4 + ((size_t)HALO_EMAX + 4) * 2;
size_t halo_smem_bytes(int nb, int umax) {
  return (size_t)umax * 2 * 32 * halo_nb(nb) * sizeof(float2) + HALO_ENTRY_BYTES;
}
int halo_umax(int nb) {
  return (int)((HALO_SMEM_BUDGET - HALO_ENTRY_BYTES) / ((size_t)2 * 32 * halo_nb(nb) * sizeof(float2)));
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  else if constexpr (BYTES == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// tile descriptor: halo rows [u0, u1), owned rows [r0, r1), entries [e0, e1)
struct TileDesc {
  int u0, u1, r0, r1, e0, e1;
};
__device__ __forceinline__ TileDesc tile_desc(const HaloArgs& h, int tau) {
  return TileDesc{__ldg(h.u0 + tau), __ldg(h.u0 + tau + 1), __ldg(h.t_r0 + tau),
                  __ldg(h.t_r0 + tau + 1), __ldg(h.e0 + tau), __ldg(h.e0 + tau + 1)};
}

template <int NBL, int NB, bool TRANSF, bool CONJ>
__global__ void __launch_bounds__(256, 2) k_spmm_halo(OpArgs op, HaloArgs h, const float2* __restrict__ z,
                                                      float2* __restrict__ pA, float2* __restrict__ pB,
                                                      float2* __restrict__ x, float2* __restrict__ q,
                                                      KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  extern __shared__ float4 sh4_[];
  float2* sz = reinterpret_cast<float2*>(sh4_);     // [umax][NB][32]: z, then p = z + beta p_prev
  float2* spv = sz + h.umax * NB * 32;               // [umax][NB][32]: p_prev
  float4* spk = reinterpret_cast<float4*>(spv + h.umax * NB * 32);  // [HALO_EMAX] planes
  float* smd = reinterpret_cast<float*>(spk + HALO_EMAX);           // [HALO_EMAX] MD
  uint32_t* sli = reinterpret_cast<uint32_t*>(smd + HALO_EMAX);     // local indices, 2 per word
  constexpr int NSPLIT = NBL / NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.y / NSPLIT, part = blockIdx.y % NSPLIT;
  const int r0 = (tile * 32 + lane) * NBL + part * NB;     // first system of this lane
  const int c0 = tile * 32 * NBL + lane + 32 * part * NB;  // its first column (stride 32)
  const bool on = r0 < op.R;
  const int par = *ks.par;
  const float2* __restrict__ src = par ? pB : pA;
  float2* __restrict__ dst = par ? pA : pB;
  BT_SEG_BEGIN(op.sp);
  (void)sr0_;
  (void)sr1_;
  LaneCoef<NB> lc;
  lane_coef<NB>(op, sg_, on ? r0 : 0, ks.active, lc);
  bool act[NB], pend[NB], usep[NB];
  float2 beta[NB], alp[NB];
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int s = sg_ * op.R + r0 + b;
    act[b] = on && lc.act[b];
    pend[b] = on && (r0 + b < op.R) && ks.pend[s] != 0;
    beta[b] = act[b] ? make_float2((float)ks.beta[2 * s], (float)ks.beta[2 * s + 1]) : make_float2(0.f, 0.f);
    alp[b] = pend[b] ? make_float2((float)ks.alpha[2 * s], (float)ks.alpha[2 * s + 1]) : make_float2(0.f, 0.f);
    usep[b] = act[b] && (beta[b].x != 0.f || beta[b].y != 0.f);
    any |= act[b] || pend[b];
  }
  const float qx = (float)lc.qx, qy = (float)lc.qy, qz = (float)lc.qz, ca = (float)lc.a;
  float cb[NB], cc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    cb[b] = (float)lc.b[b];
    cc[b] = (float)lc.c[b];
  }
  double2 acc[NB];
  float2 accf[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b] = make_double2(0, 0);
    accf[b] = make_float2(0.f, 0.f);
  }
  int cnt = 0;
  if (__syncthreads_or(any)) {
    const int tb = h.seg_tile0[sg_], te = h.seg_tile0[sg_ + 1];
    int tau = tb + sk_;
    TileDesc cur = tau < te ? tile_desc(h, tau) : TileDesc{0, 0, 0, 0, 0, 0};
    // halo rows of this warp (w, w + 8, ...): <= 32 since umax <= 256
    int myrows = cur.u1 - cur.u0 > warp ? (cur.u1 - cur.u0 - warp + 7) / 8 : 0;
    uint32_t wl = lane < myrows ? __ldg(h.ucol + cur.u0 + warp + 8 * lane) : 0u;
    for (; tau < te; tau += snb_) {
      // ---- 1. asynchronous copies: z and p_prev of the halo rows, the tile's entries
      for (int k = 0; k < myrows; ++k) {
        const uint32_t w = __shfl_sync(0xffffffffu, wl, k);
        const int uu = warp + 8 * k;
        const size_t e = (size_t)(w & 0x7FFFFFFFu) * op.Rp + c0;
        const bool own = (w >> 31) != 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (act[b]) cp_async<8>(sz + (uu * NB + b) * 32 + lane, z + e + 32 * b);
          if (usep[b] || (own && pend[b])) cp_async<8>(spv + (uu * NB + b) * 32 + lane, src + e + 32 * b);
        }
      }
      const int ne = cur.e1 - cur.e0;  // <= HALO_EMAX (tile builder)
      for (int t = threadIdx.x; t < ne; t += blockDim.x) {
        cp_async<16>(spk + t, h.pkt + cur.e0 + t);
        if constexpr (TRANSF) cp_async<4>(smd + t, h.mdt + cur.e0 + t);
      }
      const int w0 = cur.e0 >> 1, nw = ((cur.e1 + 1) >> 1) - w0;  // the index array is padded
      for (int t = threadIdx.x; t < nw; t += blockDim.x)
        cp_async<4>(sli + t, reinterpret_cast<const uint32_t*>(h.lidx) + w0 + t);
      const int loff = cur.e0 & 1;
      // owned rows of this warp (lane-parallel metadata; used after the barrier)
      const int nown = cur.r1 - cur.r0 > warp ? (cur.r1 - cur.r0 - warp + 7) / 8 : 0;  // <= 16
      const int ko = cur.r0 + warp + 8 * lane;
      const int m_row = lane < nown ? __ldg(h.rows + ko) : 0;
      const int m_e0 = lane < nown ? __ldg(h.rowe + ko) - cur.e0 : 0;
      const int m_e1 = lane < nown ? __ldg(h.rowe + ko + 1) - cur.e0 : 0;
      const int m_lo = lane < nown ? (int)__ldg(h.rowl + ko) : 0;
      // next tile's descriptor while the copies are in flight
      const bool more = tau + snb_ < te;
      const TileDesc nxt = more ? tile_desc(h, tau + snb_) : cur;
      cp_async_wait_all();
      // p = z + beta p_prev in place; each thread converts exactly what it copied
      for (int k = 0; k < myrows; ++k) {
        const int uu = warp + 8 * k;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int ix = (uu * NB + b) * 32 + lane;
          float2 pn = act[b] ? sz[ix] : make_float2(0.f, 0.f);
          if (usep[b]) {
            const float2 pv = spv[ix];
            pn.x = fmaf(beta[b].x, pv.x, fmaf(-beta[b].y, pv.y, pn.x));
            pn.y = fmaf(beta[b].x, pv.y, fmaf(beta[b].y, pv.x, pn.y));
          }
          sz[ix] = pn;
        }
      }
      // next tile's halo rows (loads in flight during the sums below)
      const int myrows_n = more ? (nxt.u1 - nxt.u0 > warp ? (nxt.u1 - nxt.u0 - warp + 7) / 8 : 0) : 0;
      const uint32_t wl_n = lane < myrows_n ? __ldg(h.ucol + nxt.u0 + warp + 8 * lane) : 0u;
      __syncthreads();
      // ---- 2. q = L p for the owned rows, everything from shared memory
      const uint16_t* sl16 = reinterpret_cast<const uint16_t*>(sli) + loff;
      for (int kk = 0; kk < nown; ++kk) {
        const int row = __shfl_sync(0xffffffffu, m_row, kk);
        const int e0 = __shfl_sync(0xffffffffu, m_e0, kk), e1 = __shfl_sync(0xffffffffu, m_e1, kk);
        const int lo = __shfl_sync(0xffffffffu, m_lo, kk);
        const size_t erow = (size_t)row * op.Rp + c0;
        float2 xv[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) xv[b] = pend[b] ? x[erow + 32 * b] : make_float2(0.f, 0.f);
        float2 P[NB], Q[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) P[b] = Q[b] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int e = e0; e < e1; ++e) {
          const float4 v = spk[e];
          const int l = sl16[e];
          const float m = qx * v.y + qy * v.z + qz * v.w;
          float a0 = ca * v.x;
          float z1 = 0.f;
          if constexpr (TRANSF) z1 = smd[e];
          const float2* xs = sz + l * NB * 32 + lane;
          const float2 m2 = make_float2(m, m);
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const float2 xx = xs[32 * b];
            float c = a0;
            if constexpr (TRANSF) c = fmaf(cb[b], z1, c);
            // packed FP32 pairs (re, im): one FFMA2 per complex update
            P[b] = __ffma2_rn(make_float2(c, c), xx, P[b]);
            Q[b] = __ffma2_rn(m2, xx, Q[b]);
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const int ix = (lo * NB + b) * 32 + lane;
          if (act[b]) {
            float2 y;
            y.x = P[b].x - cc[b] * Q[b].y;
            y.y = P[b].y + cc[b] * Q[b].x;
            q[erow + 32 * b] = y;
            float2 pv = sz[ix];
            dst[erow + 32 * b] = pv;
            if constexpr (CONJ) pv.y = -pv.y;
            accf[b].x = fmaf(pv.x, y.x, fmaf(-pv.y, y.y, accf[b].x));
            accf[b].y = fmaf(pv.x, y.y, fmaf(pv.y, y.x, accf[b].y));
          }
          if (pend[b]) {
            const float2 pp = spv[ix];
            xv[b].x = fmaf(alp[b].x, pp.x, fmaf(-alp[b].y, pp.y, xv[b].x));
            xv[b].y = fmaf(alp[b].x, pp.y, fmaf(alp[b].y, pp.x, xv[b].y));
            x[erow + 32 * b] = xv[b];
          }
        }
        if (++cnt == 16) {
          cnt = 0;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            acc[b].x += (double)accf[b].x;
            acc[b].y += (double)accf[b].y;
            accf[b] = make_float2(0.f, 0.f);
          }
        }
      }
      __syncthreads();  // the next tile overwrites the staged rows and entries
      cur = nxt;
      myrows = myrows_n;
      wl = wl_n;
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b].x += (double)accf[b].x;
    acc[b].y += (double)accf[b].y;
  }
  block_partials<NB>(acc, on ? r0 : op.Rp, op.Rp, rs.part);
  if (!last_block(rs.counter, gridDim.x * gridDim.y)) return;
  if (threadIdx.x == 0 && ks.sys_iter) atomicAdd(ks.sys_iter, (unsigned long long)*ks.n_active);
  __syncthreads();
  reduce_partials(rs.part, op.sp, op.Rp, op.R, [&](int s, double2 pq) {
    count_segment_iter(ks, s, op.R);
    krylov_alpha(ks, s, pq);
    ks.pend[s] = ks.active[s];
  });
  if (threadIdx.x == 0) *ks.par = par ^ 1;
}

template <int NBL, bool TRANSF, bool CONJ>
static void halo_attr() {
  cudaFuncSetAttribute(k_spmm_halo<NBL, halo_nb(NBL), TRANSF, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       HALO_SMEM_BUDGET);
}
// raise the dynamic shared memory limit of every instance (outside any capture)
void halo_prepare() {
  halo_attr<1, false, false>(); halo_attr<1, false, true>(); halo_attr<1, true, false>(); halo_attr<1, true, true>();
  halo_attr<2, false, false>(); halo_attr<2, false, true>(); halo_attr<2, true, false>(); halo_attr<2, true, true>();
  halo_attr<4, false, false>(); halo_attr<4, false, true>(); halo_attr<4, true, false>(); halo_attr<4, true, true>();
}

template <int NBL, bool TRANSF, bool CONJ>
static void halo_t(const OpArgs& op, const HaloArgs& h, const float2* z, float2* pA, float2* pB, float2* x,
                   float2* q, const KrylovState& ks, RedScratch rs, cudaStream_t st) {
  constexpr int NB = halo_nb(NBL);
  dim3 grid(op.sp.nblk, ((op.R + 32 * NBL - 1) / (32 * NBL)) * (NBL / NB));
  k_spmm_halo<NBL, NB, TRANSF, CONJ><<<grid, 256, halo_smem_bytes(NBL, h.umax), st>>>(op, h, z, pA, pB, x, q, ks,
                                                                                       rs);
}

void launch_spmm_halo(const OpArgs& op, const HaloArgs& h, const float2* z, float2* pA, float2* pB, float2* x,
                      float2* q, const KrylovState& ks, RedScratch rs, int conj, int nb, cudaStream_t st) {
#define BT_HALO_CASE(NBV)                                                        \
  if (op.transformed) {                                                          \
    if (conj) halo_t<NBV, true, true>(op, h, z, pA, pB, x, q, ks, rs, st);       \
    else halo_t<NBV, true, false>(op, h, z, pA, pB, x, q, ks, rs, st);           \
  } else {                                                                       \
    if (conj) halo_t<NBV, false, true>(op, h, z, pA, pB, x, q, ks, rs, st);      \
    else halo_t<NBV, false, false>(op, h, z, pA, pB, x, q, ks, rs, st);          \
  }
  switch (nb) {
    case 4: BT_HALO_CASE(4) break;
    case 2: BT_HALO_CASE(2) break;
    default: BT_HALO_CASE(1) break;
  }
#undef BT_HALO_CASE
}

}  // namespace bt
