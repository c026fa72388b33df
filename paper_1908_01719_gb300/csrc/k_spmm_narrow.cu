// "Narrow" variants of the fused SpMM for few right-hand sides (R <= 4), the
// shape of the plain per-direction FP64 solve.  Lane mapping: G = 8 lanes per
// row stride over the row's nonzeros, each lane keeps all R RHS in registers,
// and the G partial sums are combined with warp shuffles.  The operator is the
// one of k_spmm.cu (each RHS builds its own direction operator m = qhat_r.Pd).
#include "bt_kernels.cuh"

namespace bt {

constexpr int NG = 8;  // lanes per row

template <int RM, bool TRANSF>
__device__ __forceinline__ void narrow_row(const OpArgs& op, int64_t row, int g, const double (&qx)[RM],
                                           const double (&qy)[RM], const double (&qz)[RM], const double* p0o,
                                           const double2* __restrict__ x, double2 (&P)[RM], double2 (&Q)[RM],
                                           double2 (&Z)[RM]) {
#pragma unroll
  for (int b = 0; b < RM; ++b) P[b] = Q[b] = Z[b] = make_double2(0, 0);
  const int k0 = op.rp[row], k1 = op.rp[row + 1];
  for (int k = k0 + g; k < k1; k += NG) {
    const int j = __ldg(op.col + k);
    const double4 v = ldg4(op.pk64 + k);
    const double p0 = p0o ? __ldg(p0o + k) : v.x;
    double z1 = 0;
    if constexpr (TRANSF) z1 = __ldg(op.p1_64 + k);
#pragma unroll
    for (int b = 0; b < RM; ++b) {
      if (b >= op.R) break;
      const double2 xv = __ldg(x + (size_t)j * op.Rp + b);
      const double m = qx[b] * v.y + qy[b] * v.z + qz[b] * v.w;
      P[b].x = fma(p0, xv.x, P[b].x);
      P[b].y = fma(p0, xv.y, P[b].y);
      Q[b].x = fma(m, xv.x, Q[b].x);
      Q[b].y = fma(m, xv.y, Q[b].y);
      if constexpr (TRANSF) {
        Z[b].x = fma(z1, xv.x, Z[b].x);
        Z[b].y = fma(z1, xv.y, Z[b].y);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < RM; ++b) {
#pragma unroll
    for (int o = NG / 2; o > 0; o >>= 1) {
      P[b].x += __shfl_xor_sync(0xffffffffu, P[b].x, o);
      P[b].y += __shfl_xor_sync(0xffffffffu, P[b].y, o);
      Q[b].x += __shfl_xor_sync(0xffffffffu, Q[b].x, o);
      Q[b].y += __shfl_xor_sync(0xffffffffu, Q[b].y, o);
      if constexpr (TRANSF) {
        Z[b].x += __shfl_xor_sync(0xffffffffu, Z[b].x, o);
        Z[b].y += __shfl_xor_sync(0xffffffffu, Z[b].y, o);
      }
    }
  }
}

// per-block partials of RM complex values per RHS: lanes g == 0 hold them;
// reduce over the block's row groups into part[blockIdx.x][b]
template <int RM>
__device__ __forceinline__ void narrow_partials(double2 (&acc)[RM], int g, int Rp, double* part) {
  __shared__ double2 sm[256 / NG][RM];
  const int grp = threadIdx.x / NG, ngrp = blockDim.x / NG;
  if (g == 0)
#pragma unroll
    for (int b = 0; b < RM; ++b) sm[grp][b] = acc[b];
  __syncthreads();
  if (threadIdx.x < RM && threadIdx.x < Rp) {
    double2 s = make_double2(0, 0);
    for (int q = 0; q < ngrp; ++q) {
      s.x += sm[q][threadIdx.x].x;
      s.y += sm[q][threadIdx.x].y;
    }
    reinterpret_cast<double2*>(part)[(size_t)blockIdx.x * Rp + threadIdx.x] = s;
  }
}

template <int RM, bool TRANSF, bool CONJ>
__global__ void __launch_bounds__(256) k_spmm_krylov_narrow(OpArgs op, const double2* __restrict__ p,
                                                            double2* __restrict__ q, KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  const int g = threadIdx.x % NG, grp = threadIdx.x / NG, ngrp = blockDim.x / NG;
  const OpCoef cf = op_coef(op, 0);
  double qx[RM], qy[RM], qz[RM], cb[RM], cc[RM];
#pragma unroll
  for (int b = 0; b < RM; ++b) {
    const int s = b < op.R ? b : 0;
    qx[b] = op.qhat[3 * s];
    qy[b] = op.qhat[3 * s + 1];
    qz[b] = op.qhat[3 * s + 2];
    const double qq = op.q[s];
    cb[b] = cf.bq2 * qq * qq;
    cc[b] = cf.cq * qq;
  }
  double2 acc[RM];
#pragma unroll
  for (int b = 0; b < RM; ++b) acc[b] = make_double2(0, 0);
  // all lanes of a warp run the same number of row iterations (shuffles)
  // round-robin chunks of ngrp rows (one per 8-lane group); the loop trip
  // count is uniform over the block so the shuffles stay converged
  for (int64_t ch = blockIdx.x; ch * ngrp < op.n; ch += gridDim.x) {
    const int64_t row = ch * ngrp + grp;
    const bool ok = row < op.n;
    const int64_t rb = ch * ngrp;
    double2 P[RM], Q[RM], Z[RM];
    narrow_row<RM, TRANSF>(op, ok ? row : rb, ok ? g : (1 << 30), qx, qy, qz, nullptr, p, P, Q, Z);
    if (ok && g == 0) {
#pragma unroll
      for (int b = 0; b < RM; ++b) {
        if (b >= op.R) break;
        double2 y;
        const double re0 = cf.a * P[b].x + (TRANSF ? cb[b] * Z[b].x : 0.0);
        const double im0 = cf.a * P[b].y + (TRANSF ? cb[b] * Z[b].y : 0.0);
        y.x = re0 - cc[b] * Q[b].y;
        y.y = im0 + cc[b] * Q[b].x;
        const size_t e = (size_t)row * op.Rp + b;
        q[e] = y;
        double2 pv = p[e];
        if constexpr (CONJ) pv.y = -pv.y;
        acc[b].x += pv.x * y.x - pv.y * y.y;
        acc[b].y += pv.x * y.y + pv.y * y.x;
      }
    }
  }
  narrow_partials<RM>(acc, g, op.Rp, rs.part);
  if (!last_block(rs.counter, gridDim.x)) return;
  reduce_partials_flat(rs.part, gridDim.x, op.Rp, op.R, [&](int s, double2 pq) { krylov_alpha(ks, s, pq); });
}

// r = op_{P0 = K+J}(u) (mode 0 of the refinement residual), FP64, R <= 4
template <int RM, bool TRANSF>
__global__ void __launch_bounds__(256) k_resid0_narrow(OpArgs op, const double2* __restrict__ u,
                                                       double2* __restrict__ r, RefineState rf, RedScratch rs) {
  if (*rf.n_active == 0) return;
  const int g = threadIdx.x % NG, grp = threadIdx.x / NG, ngrp = blockDim.x / NG;
  const OpCoef cf = op_coef(op, 0);
  double qx[RM], qy[RM], qz[RM], cb[RM], cc[RM];
#pragma unroll
  for (int b = 0; b < RM; ++b) {
    const int s = b < op.R ? b : 0;
    qx[b] = op.qhat[3 * s];
    qy[b] = op.qhat[3 * s + 1];
    qz[b] = op.qhat[3 * s + 2];
    const double qq = op.q[s];
    cb[b] = cf.bq2 * qq * qq;
    cc[b] = cf.cq * qq;
  }
  double2 acc[RM];
#pragma unroll
  for (int b = 0; b < RM; ++b) acc[b] = make_double2(0, 0);
  // round-robin chunks of ngrp rows (one per 8-lane group); the loop trip
  // count is uniform over the block so the shuffles stay converged
  for (int64_t ch = blockIdx.x; ch * ngrp < op.n; ch += gridDim.x) {
    const int64_t row = ch * ngrp + grp;
    const bool ok = row < op.n;
    const int64_t rb = ch * ngrp;
    double2 P[RM], Q[RM], Z[RM];
    narrow_row<RM, TRANSF>(op, ok ? row : rb, ok ? g : (1 << 30), qx, qy, qz, op.p0_64, u, P, Q, Z);
    if (ok && g == 0) {
#pragma unroll
      for (int b = 0; b < RM; ++b) {
        if (b >= op.R || !rf.active[b]) continue;
        const double re0 = cf.a * P[b].x + (TRANSF ? cb[b] * Z[b].x : 0.0);
        const double im0 = cf.a * P[b].y + (TRANSF ? cb[b] * Z[b].y : 0.0);
        double2 y = make_double2(re0 - cc[b] * Q[b].y, im0 + cc[b] * Q[b].x);
        const size_t e = (size_t)row * op.Rp + b;
        r[e] = y;
        double2 uv = u[e];
        acc[b].x += y.x * y.x + y.y * y.y;
        acc[b].y += uv.x * uv.x + uv.y * uv.y;
      }
    }
  }
  narrow_partials<RM>(acc, g, op.Rp, rs.part);
  if (!last_block(rs.counter, gridDim.x)) return;
  reduce_partials_flat(rs.part, gridDim.x, op.Rp, op.R, [&](int s, double2 t) { refine_finish(0, rf, s, t); });
}

static int narrow_grid(int64_t n, int sms) {
  int64_t g = (int64_t)sms * REDUCE_BLOCKS_PER_SM;
  int64_t need = (n + 256 / NG - 1) / (256 / NG);
  return (int)std::max<int64_t>(1, std::min(g, need));
}

#define BT_NARROW_R(R, ...)                                        \
  switch (R) {                                                     \
    case 1: { constexpr int RM_ = 1; __VA_ARGS__; } break;         \
    case 2: { constexpr int RM_ = 2; __VA_ARGS__; } break;         \
    default: { constexpr int RM_ = 4; __VA_ARGS__; } break;        \
  }

void launch_spmm_krylov_f64_narrow(const OpArgs& op, const double2* p, double2* q, const KrylovState& ks,
                                   RedScratch rs, int conj, int sms, cudaStream_t st) {
  const int g = narrow_grid(op.n, sms);
  BT_NARROW_R(op.R, {
    if (op.transformed) {
      if (conj) k_spmm_krylov_narrow<RM_, true, true><<<g, 256, 0, st>>>(op, p, q, ks, rs);
      else k_spmm_krylov_narrow<RM_, true, false><<<g, 256, 0, st>>>(op, p, q, ks, rs);
    } else {
      if (conj) k_spmm_krylov_narrow<RM_, false, true><<<g, 256, 0, st>>>(op, p, q, ks, rs);
      else k_spmm_krylov_narrow<RM_, false, false><<<g, 256, 0, st>>>(op, p, q, ks, rs);
    }
  })
}

void launch_resid0_narrow(const OpArgs& op, const double2* u, double2* r, const RefineState& rf, RedScratch rs,
                          int sms, cudaStream_t st) {
  const int g = narrow_grid(op.n, sms);
  BT_NARROW_R(op.R, {
    if (op.transformed) k_resid0_narrow<RM_, true><<<g, 256, 0, st>>>(op, u, r, rf, rs);
    else k_resid0_narrow<RM_, false><<<g, 256, 0, st>>>(op, u, r, rf, rs);
  })
}

}  // namespace bt
