// Halo-staged Krylov apply: the SpMM of one Jacobi COCG/CG iteration with the
// search-direction update and the deferred solution update fused in.
//
// Rows are grouped into tiles along a Morton curve of their node coordinates
// (HaloTiles, built on the host).  A block takes one tile and one slice of
// 32*NB right-hand sides:
//   1. stage: for every halo row j of the tile (the union of the tile rows'
//      columns) form p_j = z_j + beta p_prev_j for the slice and keep it in
//      shared memory; rows the tile owns also store p_j and apply the x update
//      x_j += alpha_prev p_prev_j that the previous iteration left pending;
//   2. apply: for every owned row, q_i = sum_j L_ij p_j from shared memory
//      (L_ij = a A0_ij + bq2 q_r^2 MD_ij + i cq q_r (qhat . Pd)_ij, the step
//      operator of Appendix B / Appendix A built on the fly), and the partial
//      inner product <p, q>;
//   3. the last block forms alpha = rho / <p, q>, marks the x update of every
//      active system pending and flips the p-buffer parity.
// On the Kuhn stencil a tile of ~20 rows has ~100 halo rows, so each X row is
// read ~5 times from L2 instead of ~15 times (one gather per nonzero), and all
// halo loads of a tile are independent, which hides their latency.  The
// search-direction and solution updates ride on the same loads, so the
// separate p-update kernel and the x part of the vector update disappear.
#include "bt_kernels.cuh"

namespace bt {

constexpr int HALO_SMEM_BUDGET = 96 * 1024;  // bytes of staged p per block (2 blocks / SM)

size_t halo_smem_bytes(int nb, int umax) { return (size_t)umax * 32 * nb * sizeof(float2); }

template <int NB, bool TRANSF, bool CONJ>
__global__ void __launch_bounds__(256, 2) k_spmm_halo(OpArgs op, HaloArgs h, const float2* __restrict__ z,
                                                      float2* __restrict__ pA, float2* __restrict__ pB,
                                                      float2* __restrict__ x, float2* __restrict__ q,
                                                      KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  extern __shared__ float2 sp_[];  // [umax][NB][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = (blockIdx.y * 32 + lane) * NB;  // first system of this lane
  const int c0 = blockIdx.y * 32 * NB + lane;     // its first column (stride 32)
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
    for (int tau = tb + sk_; tau < te; tau += snb_) {
      // ---- 1. stage p = z + beta p_prev for the halo rows of the slice
      const int ub = h.u0[tau], nu = h.u0[tau + 1] - ub;
      constexpr int US = 2;  // halo rows per warp trip (loads in flight: 2 US NB)
      for (int u = warp; u < nu; u += 8 * US) {
        uint32_t w[US];
        float2 zv[US][NB], pv[US][NB];
#pragma unroll
        for (int k = 0; k < US; ++k) {
          const int uu = u + 8 * k;
          w[k] = uu < nu ? __ldg(h.ucol + ub + uu) : 0u;
          const size_t e = (size_t)(w[k] & 0x7FFFFFFFu) * op.Rp + c0;
          const bool own = (w[k] >> 31) != 0;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            zv[k][b] = (uu < nu && act[b]) ? __ldg(z + e + 32 * b) : make_float2(0.f, 0.f);
            pv[k][b] = (uu < nu && (usep[b] || (own && pend[b]))) ? __ldg(src + e + 32 * b) : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int k = 0; k < US; ++k) {
          const int uu = u + 8 * k;
          if (uu >= nu) break;
          const size_t e = (size_t)(w[k] & 0x7FFFFFFFu) * op.Rp + c0;
          const bool own = (w[k] >> 31) != 0;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            float2 pn = zv[k][b];
            pn.x = fmaf(beta[b].x, pv[k][b].x, fmaf(-beta[b].y, pv[k][b].y, pn.x));
            pn.y = fmaf(beta[b].x, pv[k][b].y, fmaf(beta[b].y, pv[k][b].x, pn.y));
            sp_[(uu * NB + b) * 32 + lane] = pn;
            if (own) {
              if (act[b]) dst[e + 32 * b] = pn;
              if (pend[b]) {
                float2 xv = x[e + 32 * b];
                xv.x = fmaf(alp[b].x, pv[k][b].x, fmaf(-alp[b].y, pv[k][b].y, xv.x));
                xv.y = fmaf(alp[b].x, pv[k][b].y, fmaf(alp[b].y, pv[k][b].x, xv.y));
                x[e + 32 * b] = xv;
              }
            }
          }
        }
      }
      __syncthreads();
      // ---- 2. q = L p for the owned rows, from shared memory
      const int ra = h.t_r0[tau], rz = h.t_r0[tau + 1];
      for (int k = ra + warp; k < rz; k += 8) {
        const int row = __ldg(h.rows + k);
        const int e0 = __ldg(h.rowe + k), e1 = __ldg(h.rowe + k + 1);
        float2 P[NB], Q[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) P[b] = Q[b] = make_float2(0.f, 0.f);
        constexpr int KU = 4;
        for (int e = e0; e < e1; e += KU) {
          float4 v[KU];
          int l[KU];
          float z1[KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            const int ee = min(e + u, e1 - 1);
            v[u] = __ldg(h.pkt + ee);
            l[u] = __ldg(h.lidx + ee);
            z1[u] = TRANSF ? __ldg(h.mdt + ee) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            if (e + u >= e1) break;
            const float m = qx * v[u].y + qy * v[u].z + qz * v[u].w;
            const float a0 = ca * v[u].x;
            const float2* xs = sp_ + l[u] * NB * 32 + lane;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 xv = xs[32 * b];
              float c = a0;
              if constexpr (TRANSF) c = fmaf(cb[b], z1[u], c);
              P[b].x = fmaf(c, xv.x, P[b].x);
              P[b].y = fmaf(c, xv.y, P[b].y);
              Q[b].x = fmaf(m, xv.x, Q[b].x);
              Q[b].y = fmaf(m, xv.y, Q[b].y);
            }
          }
        }
        const float2* ps = sp_ + (int)__ldg(h.rowl + k) * NB * 32 + lane;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (!act[b]) continue;
          float2 y;
          y.x = P[b].x - cc[b] * Q[b].y;
          y.y = P[b].y + cc[b] * Q[b].x;
          q[(size_t)row * op.Rp + c0 + 32 * b] = y;
          float2 pv = ps[32 * b];
          if constexpr (CONJ) pv.y = -pv.y;
          accf[b].x = fmaf(pv.x, y.x, fmaf(-pv.y, y.y, accf[b].x));
          accf[b].y = fmaf(pv.x, y.y, fmaf(pv.y, y.x, accf[b].y));
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
      __syncthreads();  // the next tile overwrites the staged rows
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
    krylov_alpha(ks, s, pq);
    ks.pend[s] = ks.active[s];
  });
  if (threadIdx.x == 0) *ks.par = par ^ 1;
}

template <int NB, bool TRANSF, bool CONJ>
static void halo_attr() {
  cudaFuncSetAttribute(k_spmm_halo<NB, TRANSF, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       HALO_SMEM_BUDGET);
}
// raise the dynamic shared memory limit of every instance (outside any capture)
void halo_prepare() {
  halo_attr<1, false, false>(); halo_attr<1, false, true>(); halo_attr<1, true, false>(); halo_attr<1, true, true>();
  halo_attr<2, false, false>(); halo_attr<2, false, true>(); halo_attr<2, true, false>(); halo_attr<2, true, true>();
  halo_attr<4, false, false>(); halo_attr<4, false, true>(); halo_attr<4, true, false>(); halo_attr<4, true, true>();
}

template <int NB, bool TRANSF, bool CONJ>
static void halo_t(const OpArgs& op, const HaloArgs& h, const float2* z, float2* pA, float2* pB, float2* x,
                   float2* q, const KrylovState& ks, RedScratch rs, cudaStream_t st) {
  dim3 grid(op.sp.nblk, (op.R + 32 * NB - 1) / (32 * NB));
  k_spmm_halo<NB, TRANSF, CONJ><<<grid, 256, halo_smem_bytes(NB, h.umax), st>>>(op, h, z, pA, pB, x, q, ks, rs);
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
