// Refinement residuals in double-float arithmetic.
//
// GB300 executes FP64 at about 1/58 of its FP32 rate, so the FP64-grade
// residuals of the iterative refinement are carried out on the FP32 pipes with
// error-free transformations: a value is an unevaluated sum hi + lo of two
// FP32 numbers (about 48 significand bits).  Primitives (Dekker 1971; Knuth,
// TAOCP vol. 2, 4.2.2):
//   two_sum(a, b)  = (s, e) with s = fl(a + b), s + e = a + b exactly;
//   two_prod(a, b) = (p, e) with p = fl(a b), e = fma(a, b, -p), p + e = a b.
// A dot product keeps its leading part in `hi` with two_sum and gathers every
// rounding error (and the lo x hi cross terms) in an FP32 `lo` accumulator;
// its error is about (terms) * 2^-46 of the magnitude of the terms, far below
// the refinement tolerance.
//
// The operators are those of k_spmm.cu:
//   mode 0 (step start): r = (R_n - L_n) u^{n-1} = op_{P0 = K+J}(u)
//   mode 1 (correction):  u += s d;  r -= s op_{P0 = A0}(d)
// with u and r stored as {re_hi, im_hi, re_lo, im_lo} and d the FP32 solution
// of the inner solve for the right-hand side r / s.
#include "bt_kernels.cuh"

namespace bt {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// Products that feed an error-free sum are formed with __fmul_rn, which the
// compiler never contracts into an FMA with the following addition (a
// contraction would make fl(a b) differ from the p the error term assumes).
// (sh, sl) += (ah + al) * (xh + xl)
__device__ __forceinline__ void dd_acc(float& sh, float& sl, float ah, float al, float xh, float xl) {
  float p = __fmul_rn(ah, xh);
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, fmaf(al, xh, e));
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl += t + e;
}
// (sh, sl) += (ah + al) * x, x an exact FP32 number
__device__ __forceinline__ void dd_acc1(float& sh, float& sl, float ah, float al, float x) {
  float p = __fmul_rn(ah, x);
  float e = fmaf(ah, x, -p);
  e = fmaf(al, x, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl += t + e;
}
// The same accumulations on a pair (re, im) at once, with the FP32x2
// instructions of sm_100+ (__fmul2_rn, __fadd2_rn, __ffma2_rn: each component
// rounded once, never contracted): every step is the scalar error-free
// transformation above, component by component, so the packed sums equal the
// scalar ones bit for bit.  Differences a - b are formed as fma(b, -1, a),
// which rounds exactly like the subtraction.  The coefficient enters as the
// pairs ah2 = (ah, ah), nah2 = (-ah, -ah), al2 = (al, al).
// (sh, sl) += p + e with the product -p = pn given (two_sum of sh and p)
__device__ __forceinline__ void dd2_two_sum_into(float2& sh, float2& sl, float2 pn, float2 e) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __ffma2_rn(pn, m1, sh);   // sh + p
  const float2 bb = __ffma2_rn(sh, m1, s);   // s - sh
  const float2 u1 = __ffma2_rn(bb, m1, s);   // s - bb
  const float2 u2 = __ffma2_rn(u1, m1, sh);  // sh - (s - bb)
  const float2 v = __fadd2_rn(pn, bb);       // -(p - bb)
  const float2 t = __ffma2_rn(v, m1, u2);    // u2 + (p - bb)
  sh = s;
  sl = __fadd2_rn(sl, __fadd2_rn(t, e));
}
// (sh, sl) += (ah + al) * x, x a pair of exact FP32 numbers
__device__ __forceinline__ void dd2_acc1(float2& sh, float2& sl, float2 ah2, float2 nah2, float2 al2, float2 x) {
  const float2 pn = __fmul2_rn(nah2, x);  // -p, p = fl(ah x)
  float2 e = __ffma2_rn(ah2, x, pn);      // ah x - p, exact
  e = __ffma2_rn(al2, x, e);              // + al x
  dd2_two_sum_into(sh, sl, pn, e);
}
// (sh, sl) += (ah + al) * (xh + xl), x a pair of double-float numbers
__device__ __forceinline__ void dd2_acc(float2& sh, float2& sl, float2 ah2, float2 nah2, float2 al2, float2 xh,
                                        float2 xl) {
  const float2 pn = __fmul2_rn(nah2, xh);
  float2 e = __ffma2_rn(ah2, xh, pn);
  e = __ffma2_rn(al2, xh, e);
  e = __ffma2_rn(ah2, xl, e);
  dd2_two_sum_into(sh, sl, pn, e);
}
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }

struct dd {
  float h, l;
};
__device__ __forceinline__ dd dd_norm(float h, float l) {
  dd r;
  fast_two_sum(h, l, r.h, r.l);
  return r;
}
__device__ __forceinline__ dd dd_split(double v) {
  dd r;
  r.h = (float)v;
  r.l = (float)(v - (double)r.h);
  return r;
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return dd_norm(p, e);
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return dd_norm(s, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.h, -a.l}; }

// NBL: columns of the layout tile per lane; NB (<= NBL): the share of them one
// thread computes (the residual's register budget keeps NB at 2 so that two
// blocks fit per SM); blockIdx.y = tile * (NBL / NB) + part.
template <int NBL, int NB, bool TRANSF, int MODE, class TX>
__global__ void __launch_bounds__(256) k_resid_df(OpArgs op, const TX* __restrict__ x, float4* __restrict__ u,
                                                  float4* __restrict__ r, RefineState rf, RedScratch rs) {
  if (*rf.n_active == 0) return;
  constexpr int NSPLIT = NBL / NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int tile = blockIdx.y / NSPLIT, part = blockIdx.y % NSPLIT;
  const int r0 = (tile * 32 + lane) * NBL + part * NB;
  const int c0 = tile * 32 * NBL + lane + 32 * part * NB;
  const bool on = r0 < op.R;
  LaneCoef<NB> lc;
  BT_SEG_BEGIN(op.sp);
  lane_coef<NB>(op, sg_, on ? r0 : 0, rf.active, lc);
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) any |= (on && lc.act[b]);
  const bool warp_any = __any_sync(0xffffffffu, any);
  const dd qx = dd_split(lc.qx), qy = dd_split(lc.qy), qz = dd_split(lc.qz);
  const dd ca = dd_split(lc.a);
  dd cb[NB], cc[NB];
  float sc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    cb[b] = dd_split(lc.b[b]);
    cc[b] = dd_split(lc.c[b]);
    sc[b] = (MODE == 1 && on && r0 + b < op.R) ? (float)rf.scale[sg_ * op.R + r0 + b] : 1.0f;
  }
  double2 acc[NB];
  float2 accf[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b] = make_double2(0, 0);
    accf[b] = make_float2(0, 0);
  }
  int cnt = 0;
  // the FP32 form of L d once every system of the warp is past its step's
  // first pass (as in k_resid_df_halo below)
  bool late = false;
  if constexpr (MODE == 1) {
    bool l = true;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (on && lc.act[b]) {
        const int s = sg_ * op.R + r0 + b;
        l = l && rf.rk2[s] <= 1e-8 * rf.r0n2[s];
      }
    late = __all_sync(0xffffffffu, l);
  }
  if (warp_any) {
    BT_FOR_SEG_CHUNKED_ROWS(row, warp, W) {
      const int k0 = op.rp[row], k1 = op.rp[row + 1];
      // accumulators: P (P0 x), Q (m x), Z (MD x); packed (re, im), hi/lo
      float2 Ph[NB], Pl[NB], Qh[NB], Ql[NB], Zh[NB], Zl[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) Ph[b] = Pl[b] = Qh[b] = Ql[b] = Zh[b] = Zl[b] = make_float2(0.f, 0.f);
      // column indices fetched lane-parallel, then DU gathers in flight
      constexpr int DU = 2;
      for (int kb = k0; kb < k1; kb += 32) {
        const int n_in = min(32, k1 - kb);
        const int jl = lane < n_in ? __ldg(op.col + kb + lane) : 0;
        for (int t = 0; t < n_in; t += DU) {
          TX xs[DU][NB];
#pragma unroll
          for (int u = 0; u < DU; ++u) {
            const int tt = t + u;
            const int j = __shfl_sync(0xffffffffu, jl, tt & 31);
            if (tt < n_in && on) {
#pragma unroll
              for (int b = 0; b < NB; ++b) xs[u][b] = __ldg(x + (size_t)j * op.Rp + c0 + 32 * b);
            }
          }
#pragma unroll
          for (int u = 0; u < DU; ++u) {
            const int k = kb + t + u;
            if (t + u >= n_in) break;
            if (MODE == 1 && late) {
              const float4 vh = __ldg(op.pkhi + k);
              const float m = fmaf(qx.h, vh.y, fmaf(qy.h, vh.z, qz.h * vh.w));
              const float2 p2 = bc(vh.x), m2 = bc(m);
              float2 md2 = make_float2(0.f, 0.f);
              if constexpr (TRANSF) md2 = bc(__ldg(op.kjmd_hi + k).y);
              if (!on) continue;
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                if constexpr (MODE == 1) {
                  const float2 xv = xs[u][b];
                  Ph[b] = __ffma2_rn(p2, xv, Ph[b]);
                  Qh[b] = __ffma2_rn(m2, xv, Qh[b]);
                  if constexpr (TRANSF) Zh[b] = __ffma2_rn(md2, xv, Zh[b]);
                }
              }
              continue;
            }
            const float4 vh = __ldg(op.pkhi + k), vl = __ldg(op.pklo + k);
            float p0h, p0l;
            float mdh = 0.f, mdl = 0.f;
            if (MODE == 0 || TRANSF) {
              const float2 kh = __ldg(op.kjmd_hi + k), kl = __ldg(op.kjmd_lo + k);
              mdh = kh.y;
              mdl = kl.y;
              if (MODE == 0) {
                p0h = kh.x;
                p0l = kl.x;
              } else {
                p0h = vh.x;
                p0l = vl.x;
              }
            } else {
              p0h = vh.x;
              p0l = vl.x;
            }
            // m = qhat . Pd in double-float
            float mh = 0.f, ml = 0.f;
            dd_acc(mh, ml, qx.h, qx.l, vh.y, vl.y);
            dd_acc(mh, ml, qy.h, qy.l, vh.z, vl.z);
            dd_acc(mh, ml, qz.h, qz.l, vh.w, vl.w);
            const dd m = dd_norm(mh, ml);
            const float2 p0h2 = bc(p0h), np0h2 = bc(-p0h), p0l2 = bc(p0l);
            const float2 mh2 = bc(m.h), nmh2 = bc(-m.h), ml2 = bc(m.l);
            if (!on) continue;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              if constexpr (MODE == 0) {
                const float4 xv = xs[u][b];
                const float2 xh = make_float2(xv.x, xv.y), xl = make_float2(xv.z, xv.w);
                dd2_acc(Ph[b], Pl[b], p0h2, np0h2, p0l2, xh, xl);
                dd2_acc(Qh[b], Ql[b], mh2, nmh2, ml2, xh, xl);
                if constexpr (TRANSF) dd2_acc(Zh[b], Zl[b], bc(mdh), bc(-mdh), bc(mdl), xh, xl);
              } else {
                const float2 xv = xs[u][b];
                dd2_acc1(Ph[b], Pl[b], p0h2, np0h2, p0l2, xv);
                dd2_acc1(Qh[b], Ql[b], mh2, nmh2, ml2, xv);
                if constexpr (TRANSF) dd2_acc1(Zh[b], Zl[b], bc(mdh), bc(-mdh), bc(mdl), xv);
              }
            }
          }
        }
      }
      if (on) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (!lc.act[b]) continue;
          const size_t e = (size_t)row * op.Rp + c0 + 32 * b;
          // y = a P + b Z + i c Q
          dd Pr = dd_norm(Ph[b].x, Pl[b].x), Pi = dd_norm(Ph[b].y, Pl[b].y);
          dd Qr = dd_norm(Qh[b].x, Ql[b].x), Qi = dd_norm(Qh[b].y, Ql[b].y);
          dd yr = dd_add(dd_mul(ca, Pr), dd_neg(dd_mul(cc[b], Qi)));
          dd yi = dd_add(dd_mul(ca, Pi), dd_mul(cc[b], Qr));
          if constexpr (TRANSF) {
            dd Zr = dd_norm(Zh[b].x, Zl[b].x), Zi = dd_norm(Zh[b].y, Zl[b].y);
            yr = dd_add(yr, dd_mul(cb[b], Zr));
            yi = dd_add(yi, dd_mul(cb[b], Zi));
          }
          if constexpr (MODE == 0) {
            r[e] = make_float4(yr.h, yi.h, yr.l, yi.l);
            const float4 uv = u[e];
            accf[b].x += yr.h * yr.h + yi.h * yi.h;
            accf[b].y += uv.x * uv.x + uv.y * uv.y;
          } else {
            // u += s d (exact product, double-float sum)
            const float2 dv = reinterpret_cast<const float2*>(x)[e];
            const float4 uv = u[e];
            dd s = dd{sc[b], 0.f};
            dd ur = dd_add(dd{uv.x, uv.z}, dd_mul(s, dd{dv.x, 0.f}));
            dd ui = dd_add(dd{uv.y, uv.w}, dd_mul(s, dd{dv.y, 0.f}));
            u[e] = make_float4(ur.h, ui.h, ur.l, ui.l);
            // r -= s y
            const float4 rv = r[e];
            dd rr = dd_add(dd{rv.x, rv.z}, dd_neg(dd_mul(s, yr)));
            dd ri = dd_add(dd{rv.y, rv.w}, dd_neg(dd_mul(s, yi)));
            r[e] = make_float4(rr.h, ri.h, rr.l, ri.l);
            accf[b].x += rr.h * rr.h + ri.h * ri.h;
          }
        }
      }
      if (++cnt == 32) {
        cnt = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          acc[b].x += (double)accf[b].x;
          acc[b].y += (double)accf[b].y;
          accf[b] = make_float2(0, 0);
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
  reduce_partials(rs.part, op.sp, op.Rp, op.R, [&](int s, double2 t) { refine_finish(MODE, rf, s, t); });
}

#define BT_DISPATCH_NB(nb, ...)                                 \
  switch (nb) {                                                 \
    case 4: { constexpr int NB_ = 4; __VA_ARGS__; } break;      \
    case 2: { constexpr int NB_ = 2; __VA_ARGS__; } break;      \
    default: { constexpr int NB_ = 1; __VA_ARGS__; } break;     \
  }

template <int NBL, int MODE, class TX>
static void resid_df_t(const OpArgs& op, const TX* x, float4* u, float4* r, const RefineState& rf, RedScratch rs,
                       int sms, cudaStream_t st) {
  constexpr int NB = NBL < 2 ? NBL : 2;
  dim3 grid(op.sp.nblk, ((op.R + 32 * NBL - 1) / (32 * NBL)) * (NBL / NB));
  if (op.transformed) k_resid_df<NBL, NB, true, MODE, TX><<<grid, 256, 0, st>>>(op, x, u, r, rf, rs);
  else k_resid_df<NBL, NB, false, MODE, TX><<<grid, 256, 0, st>>>(op, x, u, r, rf, rs);
}

void launch_resid0_df(const OpArgs& op, const float4* u, float4* r, const RefineState& rf, RedScratch rs, int nb,
                      int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, { resid_df_t<NB_, 0, float4>(op, u, const_cast<float4*>(u), r, rf, rs, sms, st); })
}

void launch_resid_sub_df(const OpArgs& op, const float2* d, float4* u, float4* r, const RefineState& rf,
                         RedScratch rs, int nb, int sms, cudaStream_t st) {
  BT_DISPATCH_NB(nb, { resid_df_t<NB_, 1, float2>(op, d, u, r, rf, rs, sms, st); })
}

// u^0 in double-float: rho of the dof's compartment (1 without an initial-condition array)
__global__ void k_fill_u_df(VecArgs va, float4* __restrict__ u, const double* __restrict__ rho) {
  size_t N = (size_t)va.n * va.Rp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
    int s = sys_of_col((int)(e % va.Rp), va.nb);
    const double v = rho ? rho[e / va.Rp] : 1.0;
    const float h = (float)v;
    u[e] = s < va.R ? make_float4(h, 0.f, (float)(v - (double)h), 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
void launch_fill_u_df(const VecArgs& va, float4* u, const double* rho, cudaStream_t st) {
  k_fill_u_df<<<1024, 256, 0, st>>>(va, u, rho);
}

}  // namespace bt

// ---------------------------------------------------------------- halo-staged variant
// The same two residuals over the halo tiles of the Krylov apply.  Per tile,
// asynchronous copies bring into shared memory the gathered vector (u in mode
// 0, d in mode 1) for the halo rows and the tile's double-float plane values
// (A0, Pd, K+J, MD as hi/lo pairs, copied into tile-entry order once per
// assembly) and local column indices; every owned row then forms its
// double-float sums from shared memory only.  Staged bytes per halo row:
// 32 NB sizeof(TX) = 512 (NB = 1 in mode 0, up to 2 in mode 1).
namespace bt {

template <int BYTES>
__device__ __forceinline__ void cp_async_tx(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  else if constexpr (BYTES == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

// staged entries: 48 B of planes and a 2-byte local index each; the index
// block is padded to a multiple of 16 bytes so the staged vector after it
// stays 16-byte aligned for 16-byte copies
constexpr int DF_LIDX_WORDS = (HALO_EMAX + 8) / 2;
constexpr size_t DF_ENTRY_BYTES = (size_t)HALO_EMAX * 48 + (size_t)DF_LIDX_WORDS * 4;
static_assert(DF_ENTRY_BYTES % 16 == 0, "staged vector must start 16-byte aligned");

template <int NBL, int NB, bool TRANSF, int MODE, class TX>
__global__ void __launch_bounds__(256, 2) k_resid_df_halo(OpArgs op, HaloArgs h, const TX* __restrict__ x,
                                                          float4* __restrict__ u, float4* __restrict__ r,
                                                          RefineState rf, RedScratch rs) {
  if (*rf.n_active == 0) return;
  extern __shared__ float4 sdf_[];
  float4* sent = sdf_;                                                  // [HALO_EMAX][3] planes
  uint32_t* sli = reinterpret_cast<uint32_t*>(sent + 3 * HALO_EMAX);   // local indices, 2 per word
  TX* xs_ = reinterpret_cast<TX*>(sli + DF_LIDX_WORDS);                 // [umax][NB][32]
  constexpr int NSPLIT = NBL / NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.y / NSPLIT, part = blockIdx.y % NSPLIT;
  const int r0 = (tile * 32 + lane) * NBL + part * NB;
  const int c0 = tile * 32 * NBL + lane + 32 * part * NB;
  const bool on = r0 < op.R;
  LaneCoef<NB> lc;
  BT_SEG_BEGIN(op.sp);
  (void)sr0_;
  (void)sr1_;
  lane_coef<NB>(op, sg_, on ? r0 : 0, rf.active, lc);
  bool act[NB];
  bool any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    act[b] = on && lc.act[b];
    any |= act[b];
  }
  const dd qx = dd_split(lc.qx), qy = dd_split(lc.qy), qz = dd_split(lc.qz);
  const dd ca = dd_split(lc.a);
  dd cb[NB], cc[NB];
  float sc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    cb[b] = dd_split(lc.b[b]);
    cc[b] = dd_split(lc.c[b]);
    sc[b] = (MODE == 1 && on && r0 + b < op.R) ? (float)rf.scale[sg_ * op.R + r0 + b] : 1.0f;
  }
  double2 acc[NB];
  float2 accf[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b] = make_double2(0, 0);
    accf[b] = make_float2(0, 0);
  }
  int cnt = 0;
  // A correction whose systems are all past the first pass of their step
  // (|r_prev| <= 1e-4 |r_0|) forms L d with FP32 products and sums: the
  // correction is then at most 1e-4 |r_0|, so FP32 rounding of L d (about
  // 1e-7 of sum |L_ij| |d_j|) stays near 1e-10 |r_0|, two orders below the
  // refinement tolerance; the updates of u and r stay double-float.  Every
  // warp of a block covers the same systems, so the choice is block-uniform.
  bool late = false;
  if constexpr (MODE == 1) {
    bool l = true;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (act[b]) {
        const int s = sg_ * op.R + r0 + b;
        l = l && rf.rk2[s] <= 1e-8 * rf.r0n2[s];
      }
    late = __all_sync(0xffffffffu, l);
  }
  if (__syncthreads_or(any)) {
    const int tb = h.seg_tile0[sg_], te = h.seg_tile0[sg_ + 1];
    for (int tau = tb + sk_; tau < te; tau += snb_) {
      const int ub = __ldg(h.u0 + tau), nu = __ldg(h.u0 + tau + 1) - ub;
      const int ra = __ldg(h.t_r0 + tau), rz = __ldg(h.t_r0 + tau + 1);
      const int te0 = __ldg(h.e0 + tau), te1 = __ldg(h.e0 + tau + 1);
      // ---- asynchronous copies: the gathered vector of the halo rows (active
      // lanes only; the others are never read) and the tile's entries
      const int myrows = nu > warp ? (nu - warp + 7) / 8 : 0;  // <= 32 since umax <= 256
      const uint32_t wl = lane < myrows ? __ldg(h.ucol + ub + warp + 8 * lane) : 0u;
      for (int k = 0; k < myrows; ++k) {
        const uint32_t w = __shfl_sync(0xffffffffu, wl, k);
        const int uu = warp + 8 * k;
        const size_t e = (size_t)(w & 0x7FFFFFFFu) * op.Rp + c0;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (act[b]) cp_async_tx<sizeof(TX)>(xs_ + (uu * NB + b) * 32 + lane, x + e + 32 * b);
      }
      const int ne = te1 - te0;  // <= HALO_EMAX (tile builder)
      for (int t = threadIdx.x; t < 3 * ne; t += blockDim.x) cp_async_tx<16>(sent + t, h.dft + 3 * (size_t)te0 + t);
      const int w0 = te0 >> 1, nw = ((te1 + 1) >> 1) - w0;  // the index array is padded
      for (int t = threadIdx.x; t < nw; t += blockDim.x)
        cp_async_tx<4>(sli + t, reinterpret_cast<const uint32_t*>(h.lidx) + w0 + t);
      const uint16_t* sl16 = reinterpret_cast<const uint16_t*>(sli) + (te0 & 1);
      const int nown = rz - ra > warp ? (rz - ra - warp + 7) / 8 : 0;  // <= 16
      const int ko = ra + warp + 8 * lane;
      const int m_row = lane < nown ? __ldg(h.rows + ko) : 0;
      const int m_e0 = lane < nown ? __ldg(h.rowe + ko) - te0 : 0;
      const int m_e1 = lane < nown ? __ldg(h.rowe + ko + 1) - te0 : 0;
      const int m_lo = lane < nown ? (int)__ldg(h.rowl + ko) : 0;
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
      // ---- double-float sums of the owned rows, from shared memory
      for (int kk = 0; kk < nown; ++kk) {
        const int row = __shfl_sync(0xffffffffu, m_row, kk);
        const int e0 = __shfl_sync(0xffffffffu, m_e0, kk), e1 = __shfl_sync(0xffffffffu, m_e1, kk);
        const int lo = __shfl_sync(0xffffffffu, m_lo, kk);
        float2 Ph[NB], Pl[NB], Qh[NB], Ql[NB], Zh[NB], Zl[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) Ph[b] = Pl[b] = Qh[b] = Ql[b] = Zh[b] = Zl[b] = make_float2(0.f, 0.f);
        if (MODE == 1 && late) {
          // FP32 products and sums into the high words (the low words stay 0)
          for (int e = e0; e < e1; ++e) {
            const float4 vh = sent[3 * e];
            const int l = sl16[e];
            const float m = fmaf(qx.h, vh.y, fmaf(qy.h, vh.z, qz.h * vh.w));
            const float2 p2 = bc(vh.x), m2 = bc(m);
            float2 md2 = make_float2(0.f, 0.f);
            if constexpr (TRANSF) md2 = bc(sent[3 * e + 2].y);
            const TX* xp = xs_ + l * NB * 32 + lane;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              if constexpr (MODE == 1) {
                const float2 xv = xp[32 * b];
                Ph[b] = __ffma2_rn(p2, xv, Ph[b]);
                Qh[b] = __ffma2_rn(m2, xv, Qh[b]);
                if constexpr (TRANSF) Zh[b] = __ffma2_rn(md2, xv, Zh[b]);
              }
            }
          }
        } else
        for (int e = e0; e < e1; ++e) {
          const float4 vh = sent[3 * e], vl = sent[3 * e + 1], kk4 = sent[3 * e + 2];  // {kh.x, kh.y, kl.x, kl.y}
          const int l = sl16[e];
          float p0h, p0l;
          const float mdh = kk4.y, mdl = kk4.w;
          if (MODE == 0) {
            p0h = kk4.x;
            p0l = kk4.z;
          } else {
            p0h = vh.x;
            p0l = vl.x;
          }
          float mh = 0.f, ml = 0.f;
          dd_acc(mh, ml, qx.h, qx.l, vh.y, vl.y);
          dd_acc(mh, ml, qy.h, qy.l, vh.z, vl.z);
          dd_acc(mh, ml, qz.h, qz.l, vh.w, vl.w);
          const dd m = dd_norm(mh, ml);
          const float2 p0h2 = bc(p0h), np0h2 = bc(-p0h), p0l2 = bc(p0l);
          const float2 mh2 = bc(m.h), nmh2 = bc(-m.h), ml2 = bc(m.l);
          const TX* xp = xs_ + l * NB * 32 + lane;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            if constexpr (MODE == 0) {
              const float4 xv = xp[32 * b];
              const float2 xh = make_float2(xv.x, xv.y), xl = make_float2(xv.z, xv.w);
              dd2_acc(Ph[b], Pl[b], p0h2, np0h2, p0l2, xh, xl);
              dd2_acc(Qh[b], Ql[b], mh2, nmh2, ml2, xh, xl);
              if constexpr (TRANSF) dd2_acc(Zh[b], Zl[b], bc(mdh), bc(-mdh), bc(mdl), xh, xl);
            } else {
              const float2 xv = xp[32 * b];
              dd2_acc1(Ph[b], Pl[b], p0h2, np0h2, p0l2, xv);
              dd2_acc1(Qh[b], Ql[b], mh2, nmh2, ml2, xv);
              if constexpr (TRANSF) dd2_acc1(Zh[b], Zl[b], bc(mdh), bc(-mdh), bc(mdl), xv);
            }
          }
        }
        const TX* xo = xs_ + lo * NB * 32 + lane;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (!act[b]) continue;
          const size_t e = (size_t)row * op.Rp + c0 + 32 * b;
          dd Pr = dd_norm(Ph[b].x, Pl[b].x), Pi = dd_norm(Ph[b].y, Pl[b].y);
          dd Qr = dd_norm(Qh[b].x, Ql[b].x), Qi = dd_norm(Qh[b].y, Ql[b].y);
          dd yr = dd_add(dd_mul(ca, Pr), dd_neg(dd_mul(cc[b], Qi)));
          dd yi = dd_add(dd_mul(ca, Pi), dd_mul(cc[b], Qr));
          if constexpr (TRANSF) {
            dd Zr = dd_norm(Zh[b].x, Zl[b].x), Zi = dd_norm(Zh[b].y, Zl[b].y);
            yr = dd_add(yr, dd_mul(cb[b], Zr));
            yi = dd_add(yi, dd_mul(cb[b], Zi));
          }
          if constexpr (MODE == 0) {
            r[e] = make_float4(yr.h, yi.h, yr.l, yi.l);
            const float4 uv = xo[32 * b];  // own row of u, staged
            accf[b].x += yr.h * yr.h + yi.h * yi.h;
            accf[b].y += uv.x * uv.x + uv.y * uv.y;
          } else {
            const float2 dv = xo[32 * b];  // own row of d, staged
            const float4 uv = u[e];
            dd s = dd{sc[b], 0.f};
            dd ur = dd_add(dd{uv.x, uv.z}, dd_mul(s, dd{dv.x, 0.f}));
            dd ui = dd_add(dd{uv.y, uv.w}, dd_mul(s, dd{dv.y, 0.f}));
            u[e] = make_float4(ur.h, ui.h, ur.l, ui.l);
            const float4 rv = r[e];
            dd rr = dd_add(dd{rv.x, rv.z}, dd_neg(dd_mul(s, yr)));
            dd ri = dd_add(dd{rv.y, rv.w}, dd_neg(dd_mul(s, yi)));
            r[e] = make_float4(rr.h, ri.h, rr.l, ri.l);
            accf[b].x += rr.h * rr.h + ri.h * ri.h;
          }
        }
        if (++cnt == 16) {
          cnt = 0;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            acc[b].x += (double)accf[b].x;
            acc[b].y += (double)accf[b].y;
            accf[b] = make_float2(0, 0);
          }
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc[b].x += (double)accf[b].x;
    acc[b].y += (double)accf[b].y;
  }
  block_partials<NB>(acc, on ? r0 : op.Rp, op.Rp, rs.part);
  if (!last_block(rs.counter, gridDim.x * gridDim.y)) return;
  reduce_partials(rs.part, op.sp, op.Rp, op.R, [&](int s, double2 t) { refine_finish(MODE, rf, s, t); });
}

// columns per lane one block handles: 512 staged bytes per halo row
template <int NBL, int MODE>
constexpr int df_halo_nb() {
  return MODE == 0 ? 1 : (NBL < 2 ? NBL : 2);
}

template <int NBL, int MODE, class TX>
static void resid_df_halo_t(const OpArgs& op, const HaloArgs& h, const TX* x, float4* u, float4* r,
                            const RefineState& rf, RedScratch rs, cudaStream_t st) {
  constexpr int NB = df_halo_nb<NBL, MODE>();
  dim3 grid(op.sp.nblk, ((op.R + 32 * NBL - 1) / (32 * NBL)) * (NBL / NB));
  const size_t smem = DF_ENTRY_BYTES + (size_t)h.umax * 32 * NB * sizeof(TX);
  if (op.transformed)
    k_resid_df_halo<NBL, NB, true, MODE, TX><<<grid, 256, smem, st>>>(op, h, x, u, r, rf, rs);
  else
    k_resid_df_halo<NBL, NB, false, MODE, TX><<<grid, 256, smem, st>>>(op, h, x, u, r, rf, rs);
}

template <int NBL, int MODE, class TX>
static void df_halo_attr() {
  constexpr int NB = df_halo_nb<NBL, MODE>();
  cudaFuncSetAttribute(k_resid_df_halo<NBL, NB, true, MODE, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       HALO_SMEM_BUDGET);
  cudaFuncSetAttribute(k_resid_df_halo<NBL, NB, false, MODE, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       HALO_SMEM_BUDGET);
}
void resid_df_halo_prepare() {
  df_halo_attr<4, 0, float4>();
  df_halo_attr<2, 0, float4>();
  df_halo_attr<4, 1, float2>();
  df_halo_attr<2, 1, float2>();
  df_halo_attr<1, 1, float2>();
}

// the double-float planes in tile-entry order: 3 float4 per entry
// {pkhi}, {pklo}, {kjmd_hi.x, kjmd_hi.y, kjmd_lo.x, kjmd_lo.y}
__global__ void k_gather_tile_df(const int32_t* __restrict__ slot, int64_t nnz, const float4* __restrict__ pkhi,
                                 const float4* __restrict__ pklo, const float2* __restrict__ kh,
                                 const float2* __restrict__ kl, float4* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sl = slot[k];
    out[3 * k] = pkhi[sl];
    out[3 * k + 1] = pklo[sl];
    const float2 a = kh[sl], b = kl[sl];
    out[3 * k + 2] = make_float4(a.x, a.y, b.x, b.y);
  }
}
void launch_gather_tile_df(const int32_t* slot, int64_t nnz, const float4* pkhi, const float4* pklo, const float2* kh,
                           const float2* kl, float4* out, cudaStream_t st) {
  k_gather_tile_df<<<1024, 256, 0, st>>>(slot, nnz, pkhi, pklo, kh, kl, out);
}

// mode 0 at one column per lane would need 2 x 512 staged bytes per halo row
// at the doubled umax of that layout: it stays on the row kernel
bool resid_df_halo_available(int nb, int mode) { return !(mode == 0 && nb == 1); }

void launch_resid0_df_halo(const OpArgs& op, const HaloArgs& h, const float4* u, float4* r, const RefineState& rf,
                           RedScratch rs, int nb, cudaStream_t st) {
  if (nb == 4) resid_df_halo_t<4, 0, float4>(op, h, u, const_cast<float4*>(u), r, rf, rs, st);
  else resid_df_halo_t<2, 0, float4>(op, h, u, const_cast<float4*>(u), r, rf, rs, st);
}

void launch_resid_sub_df_halo(const OpArgs& op, const HaloArgs& h, const float2* d, float4* u, float4* r,
                              const RefineState& rf, RedScratch rs, int nb, cudaStream_t st) {
  if (nb == 4) resid_df_halo_t<4, 1, float2>(op, h, d, u, r, rf, rs, st);
  else if (nb == 2) resid_df_halo_t<2, 1, float2>(op, h, d, u, r, rf, rs, st);
  else resid_df_halo_t<1, 1, float2>(op, h, d, u, r, rf, rs, st);
}

}  // namespace bt
