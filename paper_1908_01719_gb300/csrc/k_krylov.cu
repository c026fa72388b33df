// Batched Krylov vector kernels: every right-hand side (system) has its own
// scalars, convergence test and freeze mask.  Lab frame: COCG (the step matrix
// is complex symmetric, unconjugated inner products); transformed frame: CG
// (the step matrix is Hermitian positive definite).  Jacobi preconditioner
// z = diag(L_n)^-1 r with diag(L_n) = A0_ii + b_s MD_ii + i c_s (qhat.Pd)_ii
// formed on the fly.  Inner products: FP32 products summed over at most 32
// rows per thread, all further accumulation in FP64, and the block partials
// reduced by the last block in a fixed order (deterministic).
#include <algorithm>
#include "bt_kernels.cuh"

namespace bt {

// thread -> fixed set of RHS columns, rows strided by rows_per_pass
struct ElemMap {
  int RS, rpp, NK;
  __device__ ElemMap(int Rp) {
    RS = Rp < 256 ? Rp : 256;
    rpp = 256 / RS;
    NK = (Rp + 255) / 256;
  }
};
constexpr int EM_NK = 4;  // Rp <= 1024

// diag(L) for system s at row i (FP32 / FP64)
__device__ __forceinline__ float2 diag_f32(const VecArgs& va, const OpArgs& op, int64_t i, float b, float c,
                                           float qx, float qy, float qz) {
  float4 d = va.diag32[i];
  float re = d.x;
  if (op.transformed) re = fmaf(b, va.diag_md32[i], re);
  float im = c * (qx * d.y + qy * d.z + qz * d.w);
  return make_float2(re, im);
}
__device__ __forceinline__ double2 diag_f64(const VecArgs& va, const OpArgs& op, int64_t i, double b, double c,
                                            double qx, double qy, double qz) {
  double4 d = va.diag64[i];
  double re = d.x;
  if (op.transformed) re = fma(b, va.diag_md64[i], re);
  double im = c * (qx * d.y + qy * d.z + qz * d.w);
  return make_double2(re, im);
}

struct SysCoef {
  double b, c, qx, qy, qz;
};
__device__ __forceinline__ SysCoef sys_coef(const OpArgs& op, int s) {
  const OpCoef cf = op_coef(op, s / op.R);
  double q = op.q[s];
  SysCoef sc;
  sc.b = cf.bq2 * q * q;
  sc.c = cf.cq * q;
  sc.qx = op.qhat[3 * s];
  sc.qy = op.qhat[3 * s + 1];
  sc.qz = op.qhat[3 * s + 2];
  return sc;
}

// Reduce per-thread partials (NC complex pairs per RHS column) to
// part[blockIdx.x][r][NC] and return whether this block is the last one.
template <int NC>
__device__ bool elem_block_reduce(double2 (&acc)[EM_NK][NC], const ElemMap& em, int Rp, int nb, double* part,
                                  unsigned int* counter) {
  __shared__ double2 sm[256][NC];
  const int t = threadIdx.x;
  if (em.NK == 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) sm[t][c] = acc[0][c];
    __syncthreads();
    if (t < em.RS) {
      for (int c = 0; c < NC; ++c) {
        double2 s = make_double2(0, 0);
        for (int o = 0; o < em.rpp; ++o) {
          s.x += sm[o * em.RS + t][c].x;
          s.y += sm[o * em.RS + t][c].y;
        }
        reinterpret_cast<double2*>(part)[((size_t)blockIdx.x * Rp + sys_of_col(t, nb)) * NC + c] = s;
      }
    }
  } else {
    for (int k = 0; k < em.NK; ++k) {
      int r = t + 256 * k;
      if (r < Rp)
        for (int c = 0; c < NC; ++c)
          reinterpret_cast<double2*>(part)[((size_t)blockIdx.x * Rp + sys_of_col(r, nb)) * NC + c] = acc[k][c];
    }
  }
  return last_block(counter, gridDim.x);
}

static int elem_grid(const VecArgs& va) { return va.sp.nblk; }

// rows of this block: a contiguous share of its segment
#define BT_SEG_ROWS(va)                                                   \
  BT_SEG_BEGIN((va).sp);                                                  \
  const int64_t per = (sr1_ - sr0_ + snb_ - 1) / snb_;                    \
  const int64_t rb = sr0_ + (int64_t)sk_ * per, re = min(sr1_, rb + per);

// load the refinement residual (FP64 or double-float) of one element
__device__ __forceinline__ double2 load_res(const double2* p, size_t e) { return p[e]; }
__device__ __forceinline__ double2 load_res(const float4* p, size_t e) {
  float4 v = p[e];
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// ---------------------------------------------------------------- init
// r = r_res / scale_s, x = 0, z = r / diag, p = z; rho = <r, z>, |r|^2.
template <class T, class T2, class TR, bool CONJ>
__global__ void __launch_bounds__(256) k_krylov_init(OpArgs op, VecArgs va, const TR* __restrict__ rres,
                                                     const double* __restrict__ scale, const int* __restrict__ ref_active,
                                                     T2* __restrict__ x, T2* __restrict__ r, T2* __restrict__ p,
                                                     KrylovState ks, double tol, RedScratch rs) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][2];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = acc[k][1] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int rl = sys_of_col(col, va.nb);
      if (rl >= va.R) continue;
      const int s = sg_ * va.R + rl;
      const bool act = ref_active[s] != 0;
      const SysCoef sc = sys_coef(op, s);
      const double inv = (scale && act && scale[s] > 0) ? 1.0 / scale[s] : 1.0;
      T2 ar = {0, 0}, an = {0, 0};
      int cnt = 0;
      // four rows per trip, all loads issued before the arithmetic
      for (int64_t i0 = rb + ro; i0 < re; i0 += 4 * em.rpp) {
        double2 v[4];
        T2 d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          v[u] = make_double2(0, 0);
          d[u] = T2{1, 0};
          if (i < re && act) {
            v[u] = load_res(rres, (size_t)i * va.Rp + col);
            if constexpr (sizeof(T) == 4) {
              float2 df = diag_f32(va, op, i, (float)sc.b, (float)sc.c, (float)sc.qx, (float)sc.qy, (float)sc.qz);
              d[u].x = df.x; d[u].y = df.y;
            } else {
              double2 dd = diag_f64(va, op, i, sc.b, sc.c, sc.qx, sc.qy, sc.qz);
              d[u].x = dd.x; d[u].y = dd.y;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i >= re) break;
          const size_t e = (size_t)i * va.Rp + col;
          T2 rv = {0, 0}, z = {0, 0};
          if (act) {
            rv.x = (T)(v[u].x * inv);
            rv.y = (T)(v[u].y * inv);
            T den = (T)1 / (d[u].x * d[u].x + d[u].y * d[u].y);
            z.x = (rv.x * d[u].x + rv.y * d[u].y) * den;
            z.y = (rv.y * d[u].x - rv.x * d[u].y) * den;
          }
          r[e] = rv;
          p[e] = z;
          x[e] = T2{0, 0};
          T2 rc = rv;
          if constexpr (CONJ) rc.y = -rc.y;
          ar.x += rc.x * z.x - rc.y * z.y;
          ar.y += rc.x * z.y + rc.y * z.x;
          an.x += rv.x * rv.x + rv.y * rv.y;
        }
        if (++cnt == 8) {
          cnt = 0;
          acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
          ar = T2{0, 0}; an = T2{0, 0};
        }
      }
      acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
    }
  }
  if (!elem_block_reduce<2>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, va.Rp, [](int) { return false; },
                     [&](int s, const double2 (&o)[2]) {
    ks.rho[2 * s] = o[0].x;
    ks.rho[2 * s + 1] = o[0].y;
    ks.rr0[s] = o[1].x;
    ks.rr[s] = o[1].x;
    ks.tol2[s] = tol * tol * o[1].x;
    ks.iter[s] = 0;
    ks.rr_best[s] = o[1].x;
    ks.it_best[s] = 0;
    int a = ref_active[s] && o[1].x > 0;
    if (ref_active[s] && !isfinite(o[1].x)) {
      a = 0;
      ks.status[s] = BT_ENAN;
    }
    ks.active[s] = a;
    if (a) atomicAdd(&s_cnt, 1);
  });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// ---------------------------------------------------------------- update
// x += alpha p; r -= alpha q; z = r / diag; rho' = <r, z>, |r|^2; the last
// block applies the convergence test and forms beta = rho'/rho.
template <class T, class T2, bool CONJ>
__global__ void __launch_bounds__(256) k_krylov_update(OpArgs op, VecArgs va, T2* __restrict__ x,
                                                       T2* __restrict__ r, const T2* __restrict__ p,
                                                       const T2* __restrict__ q, KrylovState ks, RedScratch rs,
                                                       int* __restrict__ pmode) {
  if (*ks.n_active == 0) return;
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][2];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = acc[k][1] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int rl = sys_of_col(col, va.nb);
      if (rl >= va.R) continue;
      const int s = sg_ * va.R + rl;
      if (!ks.active[s]) continue;
      const SysCoef sc = sys_coef(op, s);
      const T axr = (T)ks.alpha[2 * s], axi = (T)ks.alpha[2 * s + 1];
      T2 ar = {0, 0}, an = {0, 0};
      int cnt = 0;
      // four rows per trip, all loads issued before the arithmetic
      for (int64_t i0 = rb + ro; i0 < re; i0 += 4 * em.rpp) {
        T2 pv[4], qv[4], xv[4], rv[4], d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i < re) {
            const size_t e = (size_t)i * va.Rp + col;
            pv[u] = p[e]; qv[u] = q[e]; xv[u] = x[e]; rv[u] = r[e];
            if constexpr (sizeof(T) == 4) {
              float2 df = diag_f32(va, op, i, (float)sc.b, (float)sc.c, (float)sc.qx, (float)sc.qy, (float)sc.qz);
              d[u].x = df.x; d[u].y = df.y;
            } else {
              double2 dd = diag_f64(va, op, i, sc.b, sc.c, sc.qx, sc.qy, sc.qz);
              d[u].x = dd.x; d[u].y = dd.y;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i >= re) break;
          const size_t e = (size_t)i * va.Rp + col;
          xv[u].x += axr * pv[u].x - axi * pv[u].y;
          xv[u].y += axr * pv[u].y + axi * pv[u].x;
          rv[u].x -= axr * qv[u].x - axi * qv[u].y;
          rv[u].y -= axr * qv[u].y + axi * qv[u].x;
          x[e] = xv[u];
          r[e] = rv[u];
          T den = (T)1 / (d[u].x * d[u].x + d[u].y * d[u].y);
          T2 z;
          z.x = (rv[u].x * d[u].x + rv[u].y * d[u].y) * den;
          z.y = (rv[u].y * d[u].x - rv[u].x * d[u].y) * den;
          T2 rc = rv[u];
          if constexpr (CONJ) rc.y = -rc.y;
          ar.x += rc.x * z.x - rc.y * z.y;
          ar.y += rc.x * z.y + rc.y * z.x;
          an.x += rv[u].x * rv[u].x + rv[u].y * rv[u].y;
        }
        if (++cnt == 8) {
          cnt = 0;
          acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
          ar = T2{0, 0}; an = T2{0, 0};
        }
      }
      acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
    }
  }
  if (!elem_block_reduce<2>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, va.Rp, [&](int s) { return !ks.active[s]; },
                     [&](int s, const double2 (&o)[2]) {
    if (krylov_step_finish(ks, s, o, pmode)) atomicAdd(&s_cnt, 1);
  });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// p = z + beta p for active systems (z recomputed from r)
template <class T, class T2>
__global__ void __launch_bounds__(256) k_krylov_p(OpArgs op, VecArgs va, const T2* __restrict__ r,
                                                  T2* __restrict__ p, KrylovState ks, const T2* __restrict__ zbuf,
                                                  const int* __restrict__ pmode) {
  if (*ks.n_active == 0) return;
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  if (t >= em.rpp * em.RS) return;
  const int rr = t % em.RS, ro = t / em.RS;
  BT_SEG_ROWS(va);
  for (int k = 0; k < em.NK; ++k) {
    const int col = rr + 256 * k;
    if (col >= va.Rp) continue;
    const int rl = sys_of_col(col, va.nb);
    if (rl >= va.R) continue;
    const int s = sg_ * va.R + rl;
    if (!ks.active[s]) continue;
    const SysCoef sc = sys_coef(op, s);
    const T br = (T)ks.beta[2 * s], bi = (T)ks.beta[2 * s + 1];
    const bool usez = zbuf && pmode && pmode[s];
    for (int64_t i0 = rb + ro; i0 < re; i0 += 4 * em.rpp) {
      T2 rv[4], pv[4], d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * em.rpp;
        if (i < re) {
          const size_t e = (size_t)i * va.Rp + col;
          rv[u] = r[e];
          pv[u] = p[e];
          if constexpr (sizeof(T) == 4) {
            float2 df = diag_f32(va, op, i, (float)sc.b, (float)sc.c, (float)sc.qx, (float)sc.qy, (float)sc.qz);
            d[u].x = df.x; d[u].y = df.y;
          } else {
            double2 dd = diag_f64(va, op, i, sc.b, sc.c, sc.qx, sc.qy, sc.qz);
            d[u].x = dd.x; d[u].y = dd.y;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * em.rpp;
        if (i >= re) break;
        T2 z;
        if (usez) {
          z = zbuf[(size_t)i * va.Rp + col];
        } else {
          T den = (T)1 / (d[u].x * d[u].x + d[u].y * d[u].y);
          z.x = (rv[u].x * d[u].x + rv[u].y * d[u].y) * den;
          z.y = (rv[u].y * d[u].x - rv[u].x * d[u].y) * den;
        }
        T2 np;
        np.x = z.x + br * pv[u].x - bi * pv[u].y;
        np.y = z.y + br * pv[u].y + bi * pv[u].x;
        p[(size_t)i * va.Rp + col] = np;
      }
    }
  }
}

// u += d (plain FP64 path); accumulates the final relative residual of the solve
__global__ void k_axpy_u(VecArgs va, const double2* __restrict__ d, double2* __restrict__ u, KrylovState ks,
                         RefineState rf) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  if (t >= em.rpp * em.RS) return;
  const int rr = t % em.RS, ro = t / em.RS;
  BT_SEG_ROWS(va);
  for (int k = 0; k < em.NK; ++k) {
    const int col = rr + 256 * k;
    if (col >= va.Rp) continue;
    const int rl = sys_of_col(col, va.nb);
    if (rl >= va.R) continue;
    const int s = sg_ * va.R + rl;
    if (!rf.active[s]) continue;
    for (int64_t i = rb + ro; i < re; i += em.rpp) {
      const size_t e = (size_t)i * va.Rp + col;
      double2 uv = u[e], dv = d[e];
      uv.x += dv.x;
      uv.y += dv.y;
      u[e] = uv;
    }
  }
}

// end of a plain-FP64 step: accumulate |r|/|r_0| of the solve into err
__global__ void k_finish_step(RefineState rf, KrylovState ks, int R) {
  for (int s = threadIdx.x; s < R; s += blockDim.x) {
    if (rf.active[s] && ks.rr0[s] > 0) rf.err[s] += sqrt(ks.rr[s] / ks.rr0[s]);
  }
}

// u^0: rho of the dof's compartment (1 without an initial-condition array)
__global__ void k_fill_u(VecArgs va, double2* __restrict__ u, const double* __restrict__ rho) {
  size_t N = (size_t)va.n * va.Rp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
    int s = sys_of_col((int)(e % va.Rp), va.nb);
    const double v = rho ? rho[e / va.Rp] : 1.0;
    u[e] = s < va.R ? make_double2(v, 0.0) : make_double2(0.0, 0.0);
  }
}

__global__ void k_set_int(int* p, int v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// S_s = sum_i w_i u_i (Eq. signal) in FP64
template <class TU>
__global__ void __launch_bounds__(256) k_signal(VecArgs va, const double* __restrict__ w, const TU* __restrict__ u,
                                                double* __restrict__ S, RedScratch rs) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][1];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int rl = sys_of_col(col, va.nb);
      if (rl >= va.R) continue;
      for (int64_t i = rb + ro; i < re; i += em.rpp) {
        double2 v = load_res(u, (size_t)i * va.Rp + col);
        double wi = w[i];
        acc[k][0].x = fma(wi, v.x, acc[k][0].x);
        acc[k][0].y = fma(wi, v.y, acc[k][0].y);
      }
    }
  }
  if (!elem_block_reduce<1>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  reduce_systems<1>(rs.part, va.sp, va.R, va.Rp, [](int) { return false; },
                     [&](int s, const double2 (&o)[1]) {
    S[2 * s] = o[0].x;
    S[2 * s + 1] = o[0].y;
  });
}

// ---------------------------------------------------------------- launchers
void launch_krylov_init_f32(const OpArgs& op, const VecArgs& va, const double2* r64, const double* scale,
                            const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks,
                            double tol, RedScratch rs, int conj, int sms, cudaStream_t st) {
  int g = elem_grid(va);
  if (conj) k_krylov_init<float, float2, double2, true><<<g, 256, 0, st>>>(op, va, r64, scale, ref_active, x, r, p, ks, tol, rs);
  else k_krylov_init<float, float2, double2, false><<<g, 256, 0, st>>>(op, va, r64, scale, ref_active, x, r, p, ks, tol, rs);
}
void launch_krylov_init_f32_df(const OpArgs& op, const VecArgs& va, const float4* rdf, const double* scale,
                               const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks,
                               double tol, RedScratch rs, int conj, int sms, cudaStream_t st) {
  int g = elem_grid(va);
  if (conj) k_krylov_init<float, float2, float4, true><<<g, 256, 0, st>>>(op, va, rdf, scale, ref_active, x, r, p, ks, tol, rs);
  else k_krylov_init<float, float2, float4, false><<<g, 256, 0, st>>>(op, va, rdf, scale, ref_active, x, r, p, ks, tol, rs);
}
void launch_krylov_update_f32(const OpArgs& op, const VecArgs& va, float2* x, float2* r, const float2* p,
                              const float2* q, const KrylovState& ks, RedScratch rs, int conj, int sms,
                              cudaStream_t st, int* pmode) {
  int g = elem_grid(va);
  if (conj) k_krylov_update<float, float2, true><<<g, 256, 0, st>>>(op, va, x, r, p, q, ks, rs, pmode);
  else k_krylov_update<float, float2, false><<<g, 256, 0, st>>>(op, va, x, r, p, q, ks, rs, pmode);
}
void launch_krylov_p_f32(const OpArgs& op, const VecArgs& va, const float2* r, float2* p, const KrylovState& ks,
                         int sms, cudaStream_t st, const float2* zbuf, const int* pmode) {
  k_krylov_p<float, float2><<<elem_grid(va), 256, 0, st>>>(op, va, r, p, ks, zbuf, pmode);
}
void launch_krylov_init_f64(const OpArgs& op, const VecArgs& va, const double2* r64, const int* ref_active,
                            double2* x, double2* r, double2* p, const KrylovState& ks, double tol, RedScratch rs,
                            int conj, int sms, cudaStream_t st) {
  int g = elem_grid(va);
  if (conj) k_krylov_init<double, double2, double2, true><<<g, 256, 0, st>>>(op, va, r64, nullptr, ref_active, x, r, p, ks, tol, rs);
  else k_krylov_init<double, double2, double2, false><<<g, 256, 0, st>>>(op, va, r64, nullptr, ref_active, x, r, p, ks, tol, rs);
}
void launch_krylov_update_f64(const OpArgs& op, const VecArgs& va, double2* x, double2* r, const double2* p,
                              const double2* q, const KrylovState& ks, RedScratch rs, int conj, int sms,
                              cudaStream_t st) {
  int g = elem_grid(va);
  if (conj) k_krylov_update<double, double2, true><<<g, 256, 0, st>>>(op, va, x, r, p, q, ks, rs, nullptr);
  else k_krylov_update<double, double2, false><<<g, 256, 0, st>>>(op, va, x, r, p, q, ks, rs, nullptr);
}
void launch_krylov_p_f64(const OpArgs& op, const VecArgs& va, const double2* r, double2* p,
                         const KrylovState& ks, int sms, cudaStream_t st) {
  k_krylov_p<double, double2><<<elem_grid(va), 256, 0, st>>>(op, va, r, p, ks, nullptr, nullptr);
}
void launch_axpy_u(const VecArgs& va, const double2* d, double2* u, const KrylovState& ks, const RefineState& rf,
                   int sms, cudaStream_t st) {
  k_axpy_u<<<elem_grid(va), 256, 0, st>>>(va, d, u, ks, rf);
}
void launch_finish_step(const RefineState& rf, const KrylovState& ks, int R, cudaStream_t st) {
  k_finish_step<<<1, 256, 0, st>>>(rf, ks, R);
}
void launch_fill_u(const VecArgs& va, double2* u, const double* rho, cudaStream_t st) {
  k_fill_u<<<1024, 256, 0, st>>>(va, u, rho);
}
void launch_set_int(int* p, int v, int n, cudaStream_t st) {
  k_set_int<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, st>>>(p, v, n);
}
void launch_signal(const VecArgs& va, const double* w, const double2* u, double* S, RedScratch rs, int sms,
                   cudaStream_t st) {
  k_signal<double2><<<elem_grid(va), 256, 0, st>>>(va, w, u, S, rs);
}
void launch_signal_df(const VecArgs& va, const double* w, const float4* u, double* S, RedScratch rs, int sms,
                      cudaStream_t st) {
  k_signal<float4><<<elem_grid(va), 256, 0, st>>>(va, w, u, S, rs);
}

}  // namespace bt

namespace bt {
// one column of the lane-interleaved state, rows [row0, row0 + rows), as FP64
template <class TU>
__global__ void k_extract_state(const TU* __restrict__ u, int64_t row0, int64_t rows, int Rp, int col,
                                double2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = load_res(u, (size_t)(row0 + i) * Rp + col);
}
void launch_extract_state(const void* u, int df, int64_t row0, int64_t rows, int Rp, int col, double2* out,
                          int sms, cudaStream_t st) {
  const int64_t want = (rows + 255) / 256;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  if (df) k_extract_state<float4><<<g, 256, 0, st>>>((const float4*)u, row0, rows, Rp, col, out);
  else k_extract_state<double2><<<g, 256, 0, st>>>((const double2*)u, row0, rows, Rp, col, out);
}
}  // namespace bt

namespace bt {
// mixed mode: RHS still refining after the last pass of a step did not reach tol_ref
__global__ void k_mark_ref_left(RefineState rf, KrylovState ks, int R) {
  for (int s = threadIdx.x; s < R; s += blockDim.x)
    if (rf.active[s] && ks.status[s] == BT_OK) ks.status[s] = BT_ENOCONV;
}
void launch_mark_ref_left(const RefineState& rf, const KrylovState& ks, int R, cudaStream_t st) {
  k_mark_ref_left<<<1, 256, 0, st>>>(rf, ks, R);
}
}  // namespace bt

namespace bt {
// rf_active[g R + r] = (step <= N_g): segments past their echo time stay frozen
__global__ void k_seg_active(int* act, int R, int G, int step, const int* segN) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < G * R; s += gridDim.x * blockDim.x)
    act[s] = step <= segN[s / R] ? 1 : 0;
}
void launch_seg_active(int* act, int R, int G, int step, const int* segN, cudaStream_t st) {
  k_seg_active<<<(G * R + 255) / 256, 256, 0, st>>>(act, R, G, step, segN);
}
}  // namespace bt

// ---------------------------------------------------------------- halo-tile iteration (FP32, Jacobi)
namespace bt {
// complex helpers: D z, r / D
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cdivf(float2 r, float2 d) {
  const float den = 1.0f / (d.x * d.x + d.y * d.y);
  return make_float2((r.x * d.x + r.y * d.y) * den, (r.y * d.x - r.x * d.y) * den);
}

// z = D^-1 (r_res / scale), x = 0; rho = <r, z>, |r|^2; beta = 0, no pending
// x update, p buffer parity 0.  The p buffers are not touched: the first
// apply takes p = z because beta = 0.
template <class TR, bool CONJ>
__global__ void __launch_bounds__(256) k_krylov_init_z(OpArgs op, VecArgs va, const TR* __restrict__ rres,
                                                       const double* __restrict__ scale,
                                                       const int* __restrict__ ref_active, float2* __restrict__ x,
                                                       float2* __restrict__ z, KrylovState ks, double tol,
                                                       RedScratch rs) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][2];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = acc[k][1] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int rl = sys_of_col(col, va.nb);
      if (rl >= va.R) continue;
      const int s = sg_ * va.R + rl;
      const bool act = ref_active[s] != 0;
      const SysCoef sc = sys_coef(op, s);
      const double inv = (scale && act && scale[s] > 0) ? 1.0 / scale[s] : 1.0;
      float2 ar = {0, 0}, an = {0, 0};
      int cnt = 0;
      // four rows per trip, all loads issued before the arithmetic
      for (int64_t i0 = rb + ro; i0 < re; i0 += 4 * em.rpp) {
        double2 v[4];
        float2 d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          v[u] = make_double2(0, 0);
          d[u] = make_float2(1.f, 0.f);
          if (i < re && act) {
            v[u] = load_res(rres, (size_t)i * va.Rp + col);
            d[u] = diag_f32(va, op, i, (float)sc.b, (float)sc.c, (float)sc.qx, (float)sc.qy, (float)sc.qz);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i >= re) break;
          const size_t e = (size_t)i * va.Rp + col;
          float2 rv = {0, 0}, zv = {0, 0};
          if (act) {
            rv = make_float2((float)(v[u].x * inv), (float)(v[u].y * inv));
            zv = cdivf(rv, d[u]);
          }
          z[e] = zv;
          x[e] = make_float2(0.f, 0.f);
          float2 rc = rv;
          if constexpr (CONJ) rc.y = -rc.y;
          ar.x += rc.x * zv.x - rc.y * zv.y;
          ar.y += rc.x * zv.y + rc.y * zv.x;
          an.x += rv.x * rv.x + rv.y * rv.y;
        }
        if (++cnt == 8) {
          cnt = 0;
          acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
          ar = float2{0, 0}; an = float2{0, 0};
        }
      }
      acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
    }
  }
  if (!elem_block_reduce<2>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) {
    s_cnt = 0;
    *ks.par = 0;
  }
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, va.Rp, [](int) { return false; },
                     [&](int s, const double2 (&o)[2]) {
    ks.rho[2 * s] = o[0].x;
    ks.rho[2 * s + 1] = o[0].y;
    ks.beta[2 * s] = 0;
    ks.beta[2 * s + 1] = 0;
    ks.pend[s] = 0;
    ks.rr0[s] = o[1].x;
    ks.rr[s] = o[1].x;
    ks.tol2[s] = tol * tol * o[1].x;
    ks.iter[s] = 0;
    ks.rr_best[s] = o[1].x;
    ks.it_best[s] = 0;
    int a = ref_active[s] && o[1].x > 0;
    if (ref_active[s] && !isfinite(o[1].x)) {
      a = 0;
      ks.status[s] = BT_ENAN;
    }
    ks.active[s] = a;
    if (a) atomicAdd(&s_cnt, 1);
  });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// r = D z - alpha q; z = D^-1 r; rho' = <r, z>, |r|^2; the last block applies
// the tests and forms beta (krylov_step_finish).
template <bool CONJ>
__global__ void __launch_bounds__(256) k_krylov_update_z(OpArgs op, VecArgs va, float2* __restrict__ z,
                                                         const float2* __restrict__ q, KrylovState ks,
                                                         RedScratch rs) {
  if (*ks.n_active == 0) return;
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][2];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = acc[k][1] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int rl = sys_of_col(col, va.nb);
      if (rl >= va.R) continue;
      const int s = sg_ * va.R + rl;
      if (!ks.active[s]) continue;
      const SysCoef sc = sys_coef(op, s);
      const float2 al = make_float2((float)ks.alpha[2 * s], (float)ks.alpha[2 * s + 1]);
      const float fb = (float)sc.b, fc = (float)sc.c, fx = (float)sc.qx, fy = (float)sc.qy, fz = (float)sc.qz;
      float2 ar = {0, 0}, an = {0, 0};
      int cnt = 0;
      for (int64_t i0 = rb + ro; i0 < re; i0 += 4 * em.rpp) {
        float2 zv[4], qv[4], d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i < re) {
            const size_t e = (size_t)i * va.Rp + col;
            zv[u] = z[e];
            qv[u] = __ldg(q + e);
            d[u] = diag_f32(va, op, i, fb, fc, fx, fy, fz);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + (int64_t)u * em.rpp;
          if (i >= re) break;
          float2 r = cmulf(d[u], zv[u]);
          const float2 aq = cmulf(al, qv[u]);
          r.x -= aq.x;
          r.y -= aq.y;
          const float2 zn = cdivf(r, d[u]);
          z[(size_t)i * va.Rp + col] = zn;
          float2 rc = r;
          if constexpr (CONJ) rc.y = -rc.y;
          ar.x += rc.x * zn.x - rc.y * zn.y;
          ar.y += rc.x * zn.y + rc.y * zn.x;
          an.x += r.x * r.x + r.y * r.y;
        }
        if (++cnt == 8) {
          cnt = 0;
          acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
          ar = float2{0, 0}; an = float2{0, 0};
        }
      }
      acc[k][0].x += ar.x; acc[k][0].y += ar.y; acc[k][1].x += an.x;
    }
  }
  if (!elem_block_reduce<2>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, va.Rp, [&](int s) { return !ks.active[s]; },
                     [&](int s, const double2 (&o)[2]) {
    if (krylov_step_finish(ks, s, o, nullptr)) atomicAdd(&s_cnt, 1);
  });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// x += alpha p for systems whose last apply is still pending (after the loop);
// p is the buffer the last apply wrote (the current parity's source).
__global__ void __launch_bounds__(256) k_flush_x(VecArgs va, float2* __restrict__ x, const float2* __restrict__ pA,
                                                 const float2* __restrict__ pB, KrylovState ks) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  if (t >= em.rpp * em.RS) return;
  const int rr = t % em.RS, ro = t / em.RS;
  const float2* __restrict__ p = *ks.par ? pB : pA;
  BT_SEG_ROWS(va);
  for (int k = 0; k < em.NK; ++k) {
    const int col = rr + 256 * k;
    if (col >= va.Rp) continue;
    const int rl = sys_of_col(col, va.nb);
    if (rl >= va.R) continue;
    const int s = sg_ * va.R + rl;
    if (!ks.pend[s]) continue;
    const float2 al = make_float2((float)ks.alpha[2 * s], (float)ks.alpha[2 * s + 1]);
    for (int64_t i = rb + ro; i < re; i += em.rpp) {
      const size_t e = (size_t)i * va.Rp + col;
      const float2 pv = __ldg(p + e);
      float2 xv = x[e];
      xv.x += al.x * pv.x - al.y * pv.y;
      xv.y += al.x * pv.y + al.y * pv.x;
      x[e] = xv;
    }
  }
}
// clears the pending flags once every block has flushed (separate launch)
__global__ void k_clear_pend(KrylovState ks, int n) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) ks.pend[s] = 0;
}

void launch_krylov_init_z(const OpArgs& op, const VecArgs& va, const void* rres, int df, const double* scale,
                          const int* ref_active, float2* x, float2* z, const KrylovState& ks, double tol,
                          RedScratch rs, int conj, cudaStream_t st) {
  const int g = elem_grid(va);
  if (df) {
    if (conj) k_krylov_init_z<float4, true><<<g, 256, 0, st>>>(op, va, (const float4*)rres, scale, ref_active, x, z, ks, tol, rs);
    else k_krylov_init_z<float4, false><<<g, 256, 0, st>>>(op, va, (const float4*)rres, scale, ref_active, x, z, ks, tol, rs);
  } else {
    if (conj) k_krylov_init_z<double2, true><<<g, 256, 0, st>>>(op, va, (const double2*)rres, scale, ref_active, x, z, ks, tol, rs);
    else k_krylov_init_z<double2, false><<<g, 256, 0, st>>>(op, va, (const double2*)rres, scale, ref_active, x, z, ks, tol, rs);
  }
}
void launch_krylov_update_z(const OpArgs& op, const VecArgs& va, float2* z, const float2* q, const KrylovState& ks,
                            RedScratch rs, int conj, cudaStream_t st) {
  const int g = elem_grid(va);
  if (conj) k_krylov_update_z<true><<<g, 256, 0, st>>>(op, va, z, q, ks, rs);
  else k_krylov_update_z<false><<<g, 256, 0, st>>>(op, va, z, q, ks, rs);
}
void launch_flush_x(const VecArgs& va, float2* x, const float2* pA, const float2* pB, const KrylovState& ks,
                    cudaStream_t st) {
  k_flush_x<<<elem_grid(va), 256, 0, st>>>(va, x, pA, pB, ks);
  const int n = va.sp.G * va.R;
  k_clear_pend<<<(n + 255) / 256, 256, 0, st>>>(ks, n);
}
}  // namespace bt

// ---------------------------------------------------------------- weak pseudo-periodic coupling
namespace bt {
__device__ __forceinline__ void store_res(double2* p, size_t e, double2 v) { p[e] = v; }
__device__ __forceinline__ void store_res(float4* p, size_t e, double2 v) {
  const float hr = (float)v.x, hi = (float)v.y;
  p[e] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
}

// r_i += scale sum_j w_ij e^{i sign q qhat_k L_k F_n} u_j over the partner-face
// entries of boundary row i (Appendix B, explicit partner side of the
// artificial-permeability condition), for every system (one geometry).
template <class T>
__global__ void __launch_bounds__(256) k_weak_coupling(WeakArgs wa, VecArgs va, OpArgs op, const T* __restrict__ u,
                                                       T* __restrict__ r) {
  const double F = wa.F[wa.step_dev ? *wa.step_dev : wa.step_host];
  for (int64_t k = blockIdx.x; k < wa.nr; k += gridDim.x) {
    const int row = wa.rows[k];
    const int e0 = wa.ptr[k], e1 = wa.ptr[k + 1];
    for (int c = threadIdx.x; c < va.Rp; c += blockDim.x) {
      const int s = sys_of_col(c, va.nb);
      if (s >= va.R) continue;
      const double q = op.q[s];
      double2 acc = make_double2(0, 0);
      for (int e = e0; e < e1; ++e) {
        const int code = wa.code[e];
        const int ax = code & 3;
        const double phi = ((code & 4) ? -1.0 : 1.0) * q * op.qhat[3 * s + ax] * wa.L[ax] * F;
        double sn, cs;
        sincos(phi, &sn, &cs);
        const double2 v = load_res(u, (size_t)wa.col[e] * va.Rp + c);
        acc.x += wa.w[e] * (cs * v.x - sn * v.y);
        acc.y += wa.w[e] * (cs * v.y + sn * v.x);
      }
      const size_t er = (size_t)row * va.Rp + c;
      double2 rv = load_res(r, er);
      rv.x += wa.scale * acc.x;
      rv.y += wa.scale * acc.y;
      store_res(r, er, rv);
    }
  }
}

// The step-start bookkeeping of the refinement again, after the coupling
// changed r_0: |r_0|^2 and |u|^2 per system, then refine_finish(0) with every
// system of the (single) geometry active.
template <class T>
__global__ void __launch_bounds__(256) k_resid0_renorm(VecArgs va, const T* __restrict__ u,
                                                       const T* __restrict__ r, RefineState rf, RedScratch rs) {
  ElemMap em(va.Rp);
  const int t = threadIdx.x;
  const bool live = t < em.rpp * em.RS;
  const int rr = t % em.RS, ro = t / em.RS;
  double2 acc[EM_NK][1];
  for (int k = 0; k < EM_NK; ++k) acc[k][0] = make_double2(0, 0);
  BT_SEG_ROWS(va);
  if (live) {
    for (int k = 0; k < em.NK; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      if (sys_of_col(col, va.nb) >= va.R) continue;
      for (int64_t i = rb + ro; i < re; i += em.rpp) {
        const double2 a = load_res(r, (size_t)i * va.Rp + col), b = load_res(u, (size_t)i * va.Rp + col);
        acc[k][0].x += a.x * a.x + a.y * a.y;
        acc[k][0].y += b.x * b.x + b.y * b.y;
      }
    }
  }
  if (!elem_block_reduce<1>(acc, em, va.Rp, va.nb, rs.part, rs.counter)) return;
  if (threadIdx.x == 0) *rf.n_active = va.sp.G * va.R;
  __syncthreads();
  reduce_systems<1>(rs.part, va.sp, va.R, va.Rp, [](int) { return false; },
                     [&](int s, const double2 (&o)[1]) {
    rf.active[s] = 1;
    refine_finish(0, rf, s, o[0]);
  });
}

void launch_weak_coupling(const WeakArgs& wa, const VecArgs& va, const OpArgs& op, const void* u, void* r, int df,
                          cudaStream_t st) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(wa.nr, 4096));
  if (df) k_weak_coupling<float4><<<g, 256, 0, st>>>(wa, va, op, (const float4*)u, (float4*)r);
  else k_weak_coupling<double2><<<g, 256, 0, st>>>(wa, va, op, (const double2*)u, (double2*)r);
}
void launch_resid0_renorm(const VecArgs& va, const void* u, const void* r, const RefineState& rf, RedScratch rs,
                          int df, cudaStream_t st) {
  if (df) k_resid0_renorm<float4><<<elem_grid(va), 256, 0, st>>>(va, (const float4*)u, (const float4*)r, rf, rs);
  else k_resid0_renorm<double2><<<elem_grid(va), 256, 0, st>>>(va, (const double2*)u, (const double2*)r, rf, rs);
}
}  // namespace bt
