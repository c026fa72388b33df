// Fused complex multi-right-hand-side SpMM over the shared CSR pattern.
//
// One operator for every right-hand side r (direction d(r), q_r = gamma|g_r|):
//   y_r = a (P0 x_r) + bq2 q_r^2 (P1 x_r) + i cq q_r (sum_k qhat_{d,k} Pd_k) x_r
// Lab frame (Appendix B, A = M/k - theta(-(i gamma f) J - S - I)):
//   P0 = A0 = M + theta dt (K + J), Pd = (Mx, My, Mz), cq = theta dt f_bar_n.
// Transformed frame (Appendix A, weak form F(u, v, t)):
//   P0 = A0, P1 = MD, Pd = (Ex, Ey, Ez), bq2 = theta dt F_n^2, cq = theta dt F_n.
// The direction operator m_d = qhat_d . Pd is built on the fly once per
// nonzero per lane and reused for the lane's NB right-hand sides (all of one
// direction), so the pattern and planes are read once for all RHS.
//
// Lane mapping ("wide"): grid.y tiles the RHS in groups of 32*NB; lane l owns
// RHS [r0, r0+NB), r0 = (32 blockIdx.y + l) NB; warps of a block take
// consecutive rows of the block's contiguous row range, so neighbouring rows'
// gathers of X hit L1.  X, Y are [n][Rp] interleaved complex.
#include "bt_kernels.cuh"

namespace bt {

constexpr int KU = 4;  // gathers in flight per warp

int spmm_grid_rows(int64_t n, int sms) {
  int64_t g = (int64_t)sms * REDUCE_BLOCKS_PER_SM;
  int64_t chunks = (n + ROW_CHUNK - 1) / ROW_CHUNK;
  return (int)std::max<int64_t>(1, std::min(g, chunks));
}

// ---------------------------------------------------------------- Krylov apply
// q = L p for every active RHS, plus the fused inner product <p, q>
// (unconjugated p^T q for COCG, p^H q for CG); the last block turns it into
// alpha = rho / <p, q>.
template <int NB, bool TRANSF, bool CONJ, class T, class T2, class PK>
__global__ void __launch_bounds__(256) k_spmm_krylov(OpArgs op, const T2* __restrict__ p, T2* __restrict__ q,
                                                     KrylovState ks, RedScratch rs, const PK* __restrict__ pk,
                                                     const T* __restrict__ p1) {
  if (*ks.n_active == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int r0 = (blockIdx.y * 32 + lane) * NB;     // first system of this lane
  const int c0 = blockIdx.y * 32 * NB + lane;        // its first column (stride 32)
  const bool on = r0 < op.R;
  LaneCoef<NB> lc;
  BT_SEG_BEGIN(op.sp);
  lane_coef<NB>(op, sg_, on ? r0 : 0, ks.active, lc);
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) any |= (on && lc.act[b]);
  const bool warp_any = __any_sync(0xffffffffu, any);
  const T qx = (T)lc.qx, qy = (T)lc.qy, qz = (T)lc.qz, ca = (T)lc.a;
  T cb[NB], cc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    cb[b] = (T)lc.b[b];
    cc[b] = (T)lc.c[b];
  }
  double2 acc[NB];
  T2 accf[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b] = make_double2(0, 0);
    accf[b].x = 0; accf[b].y = 0;
  }
  int cnt = 0;
  if (warp_any) {
    BT_FOR_SEG_CHUNKED_ROWS(row, warp, W) {
      const int k0 = op.rp[row], k1 = op.rp[row + 1];
      T2 P[NB], Q[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        P[b].x = 0; P[b].y = 0; Q[b].x = 0; Q[b].y = 0;
      }
      // the row's column indices are fetched lane-parallel and broadcast with
      // shuffles, so U gathers of X are in flight at once
      for (int kb = k0; kb < k1; kb += 32) {
        const int cnt = min(32, k1 - kb);
        const int jl = lane < cnt ? __ldg(op.col + kb + lane) : 0;
        for (int t = 0; t < cnt; t += KU) {
          T2 x[KU][NB];
          PK v[KU];
          T z1[KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            const int tt = t + u;
            const int j = __shfl_sync(0xffffffffu, jl, tt & 31);
            if (tt < cnt) {
              v[u] = ldg4(pk + kb + tt);
              z1[u] = TRANSF ? __ldg(p1 + kb + tt) : (T)0;
              if (on) load_x<NB>(p + (size_t)j * op.Rp + c0, x[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            if (t + u >= cnt) break;
            const T m = qx * v[u].y + qy * v[u].z + qz * v[u].w;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              T2 xb = x[u][b];
              if (!on) { xb.x = 0; xb.y = 0; }
              T c0 = ca * v[u].x;
              if constexpr (TRANSF) c0 = fma(cb[b], z1[u], c0);
              P[b].x = fma(c0, xb.x, P[b].x);
              P[b].y = fma(c0, xb.y, P[b].y);
              Q[b].x = fma(m, xb.x, Q[b].x);
              Q[b].y = fma(m, xb.y, Q[b].y);
            }
          }
        }
      }
      if (on) {
        T2 xi[NB];
        load_x<NB>(p + (size_t)row * op.Rp + c0, xi);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          T2 y;
          y.x = P[b].x - cc[b] * Q[b].y;
          y.y = P[b].y + cc[b] * Q[b].x;
          q[(size_t)row * op.Rp + c0 + 32 * b] = y;
          // <p, q>: unconjugated (COCG) or conjugated (CG)
          T2 pv = xi[b];
          if constexpr (CONJ) pv.y = -pv.y;
          accf[b].x = fma(pv.x, y.x, fma(-pv.y, y.y, accf[b].x));
          accf[b].y = fma(pv.x, y.y, fma(pv.y, y.x, accf[b].y));
        }
      }
      if (++cnt == 32) {
        cnt = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          acc[b].x += (double)accf[b].x;
          acc[b].y += (double)accf[b].y;
          accf[b].x = 0; accf[b].y = 0;
        }
      }
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
  });
}

// ---------------------------------------------------------------- plane gather
// The packed FP32 planes (and MD) in the entry order of a tiling: out[k] = in[slot[k]].
__global__ void k_gather_tile_planes(const int32_t* __restrict__ slot, int64_t nnz, const float4* __restrict__ pk32,
                                     const float* __restrict__ md32, float4* __restrict__ pkt, float* __restrict__ mdt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = slot[k];
    pkt[k] = pk32[s];
    mdt[k] = md32[s];
  }
}

void launch_gather_tile_planes(const int32_t* slot, int64_t nnz, const float4* pk32, const float* md32, float4* pkt,
                               float* mdt, cudaStream_t st) {
  k_gather_tile_planes<<<1024, 256, 0, st>>>(slot, nnz, pk32, md32, pkt, mdt);
}

template <int NB, bool TRANSF, bool CONJ>
static void spmm_krylov_f32_t(const OpArgs& op, const float2* p, float2* q, const KrylovState& ks, RedScratch rs,
                              int sms, cudaStream_t st) {
  dim3 grid(op.sp.nblk, (op.R + 32 * NB - 1) / (32 * NB));
  k_spmm_krylov<NB, TRANSF, CONJ, float, float2, float4><<<grid, 256, 0, st>>>(op, p, q, ks, rs, op.pk32, op.p1_32);
}
template <int NB, bool TRANSF, bool CONJ>
static void spmm_krylov_f64_t(const OpArgs& op, const double2* p, double2* q, const KrylovState& ks,
                              RedScratch rs, int sms, cudaStream_t st) {
  dim3 grid(op.sp.nblk, (op.R + 32 * NB - 1) / (32 * NB));
  k_spmm_krylov<NB, TRANSF, CONJ, double, double2, double4><<<grid, 256, 0, st>>>(op, p, q, ks, rs, op.pk64,
                                                                                   op.p1_64);
}

#define BT_DISPATCH_NB(nb, ...)                 \
  switch (nb) {                                 \
    case 4: { constexpr int NB_ = 4; __VA_ARGS__; } break; \
    case 2: { constexpr int NB_ = 2; __VA_ARGS__; } break; \
    default: { constexpr int NB_ = 1; __VA_ARGS__; } break; \
  }

void launch_spmm_krylov_f32(const OpArgs& op, const float2* p, float2* q, const KrylovState& ks, RedScratch rs,
                            int conj, int nb, int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, {
    if (op.transformed) {
      if (conj) spmm_krylov_f32_t<NB_, true, true>(op, p, q, ks, rs, sms, st);
      else spmm_krylov_f32_t<NB_, true, false>(op, p, q, ks, rs, sms, st);
    } else {
      if (conj) spmm_krylov_f32_t<NB_, false, true>(op, p, q, ks, rs, sms, st);
      else spmm_krylov_f32_t<NB_, false, false>(op, p, q, ks, rs, sms, st);
    }
  })
}

void launch_spmm_krylov_f64(const OpArgs& op, const double2* p, double2* q, const KrylovState& ks,
                            RedScratch rs, int conj, int nb, int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, {
    if (op.transformed) {
      if (conj) spmm_krylov_f64_t<NB_, true, true>(op, p, q, ks, rs, sms, st);
      else spmm_krylov_f64_t<NB_, true, false>(op, p, q, ks, rs, sms, st);
    } else {
      if (conj) spmm_krylov_f64_t<NB_, false, true>(op, p, q, ks, rs, sms, st);
      else spmm_krylov_f64_t<NB_, false, false>(op, p, q, ks, rs, sms, st);
    }
  })
}

// ---------------------------------------------------------------- refinement residuals (native FP64)
// MODE 0 (step start): r = op_{P0 = K+J}(u) = (R_n - L_n) u^{n-1}, partials |r|^2, |u|^2.
// MODE 1 (after an inner solve): u += s d; r -= s op_{P0 = A0}(d), partial |r|^2.
template <int NB, bool TRANSF, int MODE, class TX2>
__global__ void __launch_bounds__(256) k_resid64(OpArgs op, const TX2* __restrict__ x, double2* __restrict__ u,
                                                 double2* __restrict__ r, RefineState rf, RedScratch rs) {
  if (*rf.n_active == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int r0 = (blockIdx.y * 32 + lane) * NB;
  const int c0 = blockIdx.y * 32 * NB + lane;
  const bool on = r0 < op.R;
  LaneCoef<NB> lc;
  BT_SEG_BEGIN(op.sp);
  lane_coef<NB>(op, sg_, on ? r0 : 0, rf.active, lc);
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) any |= (on && lc.act[b]);
  const bool warp_any = __any_sync(0xffffffffu, any);
  double sc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) sc[b] = (MODE == 1 && on) ? rf.scale[sg_ * op.R + r0 + b] : 1.0;
  double2 acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = make_double2(0, 0);
  if (warp_any) {
    BT_FOR_SEG_CHUNKED_ROWS(row, warp, W) {
      const int k0 = op.rp[row], k1 = op.rp[row + 1];
      double2 P[NB], Q[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        P[b] = make_double2(0, 0);
        Q[b] = make_double2(0, 0);
      }
      for (int k = k0; k < k1; ++k) {
        const int j = __ldg(op.col + k);
        const double4 v = ldg4(op.pk64 + k);
        const double m = lc.qx * v.y + lc.qy * v.z + lc.qz * v.w;
        const double p0 = (MODE == 0) ? __ldg(op.p0_64 + k) : v.x;
        double z1 = 0;
        if constexpr (TRANSF) z1 = __ldg(op.p1_64 + k);
        if (on) {
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            TX2 xv = __ldg(x + (size_t)j * op.Rp + c0 + 32 * b);
            double xr = (double)xv.x, xim = (double)xv.y;
            double c0 = lc.a * p0;
            if constexpr (TRANSF) c0 = fma(lc.b[b], z1, c0);
            P[b].x = fma(c0, xr, P[b].x);
            P[b].y = fma(c0, xim, P[b].y);
            Q[b].x = fma(m, xr, Q[b].x);
            Q[b].y = fma(m, xim, Q[b].y);
          }
        }
      }
      if (on) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (!lc.act[b]) continue;
          const size_t e = (size_t)row * op.Rp + c0 + 32 * b;
          double2 y = make_double2(P[b].x - lc.c[b] * Q[b].y, P[b].y + lc.c[b] * Q[b].x);
          if (MODE == 0) {
            r[e] = y;
            double2 uv = u[e];
            acc[b].x += y.x * y.x + y.y * y.y;
            acc[b].y += uv.x * uv.x + uv.y * uv.y;
          } else {
            TX2 dv = x[e];
            double2 uv = u[e];
            uv.x += sc[b] * (double)dv.x;
            uv.y += sc[b] * (double)dv.y;
            u[e] = uv;
            double2 rv = r[e];
            rv.x -= sc[b] * y.x;
            rv.y -= sc[b] * y.y;
            r[e] = rv;
            acc[b].x += rv.x * rv.x + rv.y * rv.y;
          }
        }
      }
    }
  }
  block_partials<NB>(acc, on ? r0 : op.Rp, op.Rp, rs.part);
  if (!last_block(rs.counter, gridDim.x * gridDim.y)) return;
  reduce_partials(rs.part, op.sp, op.Rp, op.R, [&](int s, double2 t) { refine_finish(MODE, rf, s, t); });
}

template <int NB, bool TRANSF>
static void resid0_t(const OpArgs& op, const double2* u, double2* r, const RefineState& rf, RedScratch rs, int sms,
                     cudaStream_t st) {
  dim3 grid(op.sp.nblk, (op.R + 32 * NB - 1) / (32 * NB));
  // MODE 0 only reads u, through both pointers; restrict allows aliasing objects that are not modified
  k_resid64<NB, TRANSF, 0, double2><<<grid, 256, 0, st>>>(op, u, const_cast<double2*>(u), r, rf, rs);
}
template <int NB, bool TRANSF>
static void resid_sub_t(const OpArgs& op, const float2* d, double2* u, double2* r, const RefineState& rf,
                        RedScratch rs, int sms, cudaStream_t st) {
  dim3 grid(op.sp.nblk, (op.R + 32 * NB - 1) / (32 * NB));
  k_resid64<NB, TRANSF, 1, float2><<<grid, 256, 0, st>>>(op, d, u, r, rf, rs);
}

void launch_resid0(const OpArgs& op, const double2* u, double2* r, const RefineState& rf, RedScratch rs,
                   int nb, int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, {
    if (op.transformed) resid0_t<NB_, true>(op, u, r, rf, rs, sms, st);
    else resid0_t<NB_, false>(op, u, r, rf, rs, sms, st);
  })
}

void launch_resid_sub(const OpArgs& op, const float2* d, double2* u, double2* r, const RefineState& rf,
                      RedScratch rs, int nb, int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, {
    if (op.transformed) resid_sub_t<NB_, true>(op, d, u, r, rf, rs, sms, st);
    else resid_sub_t<NB_, false>(op, d, u, r, rf, rs, sms, st);
  })
}

}  // namespace bt
