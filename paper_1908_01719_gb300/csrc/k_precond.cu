// Learned polynomial preconditioner: BF16 MLP inference and training kernels,
// the Horner application of the polynomial inside the batched Krylov solver,
// and the residual-decay (Gram) data of step solves used for training.
//
// Model: features phi = (dt, q|f| (lab) or q|F| (transformed), D, kappa, h),
// x_k = (log(phi_k + eps_k) - mu_k) / sd_k; a1 = relu(W1 x + b1) (64),
// a2 = relu(W2 a1 + b2) (64), c = W3 a2 + b3 (9); weights and biases stored in
// bfloat16 for the forward pass, FP32 accumulation, FP32 master copy for Adam.
// Preconditioner P_c = sum_{j=0}^{8} c_j B^j D^-1, B = D^-1 L, D = diag(L),
// applied by Horner: z_8 = c_8 D^-1 r, z_j = D^-1 (c_j r + L z_{j+1}).
// Training data of one RHS r: v_0 = D^-1 r, v_{j+1} = D^-1 L v_j,
// y_j = L v_j = D v_{j+1}; G = Re(Y^H Y)/|r|^2, h = Re(Y^H r)/|r|^2, and the
// per-sample loss |r - L P_c r|^2/|r|^2 = 1 - 2 c.h + c.G c; training adds
// its spread e (2 |c|.|h| + |c|.|G| |c|) for data known to relative accuracy
// e (the Krylov basis is nearly dependent and G, h come from FP32 vectors, so
// without it the network can fit rounding instead of the operator).
#include <cuda_bf16.h>

#include "bt_kernels.cuh"

namespace bt {

// feature normalisation: eps, mu, sd per feature
__constant__ float c_fnorm[MLP_IN][3] = {
    {1e-3f, 3.9f, 0.5f}, {1e-6f, -10.0f, 2.0f}, {1e-6f, -6.2f, 0.3f}, {1e-8f, -10.4f, 0.7f}, {1e-3f, -0.5f, 0.7f}};

// parameter offsets in the flat vector: W1 (64x5), b1, W2 (64x64), b2, W3 (9x64), b3
constexpr int OW1 = 0, OB1 = OW1 + MLP_H * MLP_IN, OW2 = OB1 + MLP_H, OB2 = OW2 + MLP_H * MLP_H,
              OW3 = OB2 + MLP_H, OB3 = OW3 + MLP_OUT * MLP_H;
static_assert(OB3 + MLP_OUT == MLP_NPARAM, "parameter layout");

__device__ __forceinline__ float wbf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// One warp evaluates the network for one sample; smem holds a1, a2 of the warp.
// Returns c in lanes 0..8 (other lanes 0); z1/z2 kept for the backward pass.
struct MlpAct {
  float z1[2], z2[2];  // pre-activations of units lane, lane + 32
  float c;             // output lane < 9
};
__device__ __forceinline__ MlpAct mlp_warp(const __nv_bfloat16* __restrict__ w, const float (&x)[MLP_IN],
                                           float* sa1, float* sa2) {
  const int lane = threadIdx.x & 31;
  MlpAct a;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    float s = wbf(w, OB1 + j);
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) s = fmaf(wbf(w, OW1 + j * MLP_IN + i), x[i], s);
    a.z1[q] = s;
    sa1[j] = fmaxf(s, 0.f);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = lane + 32 * q;
    float s = wbf(w, OB2 + k);
    for (int j = 0; j < MLP_H; ++j) s = fmaf(wbf(w, OW2 + k * MLP_H + j), sa1[j], s);
    a.z2[q] = s;
    sa2[k] = fmaxf(s, 0.f);
  }
  __syncwarp();
  a.c = 0.f;
  if (lane < MLP_OUT) {
    float s = wbf(w, OB3 + lane);
    for (int k = 0; k < MLP_H; ++k) s = fmaf(wbf(w, OW3 + lane * MLP_H + k), sa2[k], s);
    a.c = s;
  }
  return a;
}

__device__ __forceinline__ void load_features(const float* __restrict__ raw, float (&x)[MLP_IN]) {
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) x[i] = (logf(raw[i] + c_fnorm[i][0]) - c_fnorm[i][1]) / c_fnorm[i][2];
}

// inference: coef[s][0..8] for S samples (raw features [S][5])
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ feat, int S, double* __restrict__ coef) {
  __shared__ float sa[8][2][MLP_H];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * 8 + warp;
  if (s >= S) return;
  float x[MLP_IN];
  load_features(feat + (size_t)MLP_IN * s, x);
  MlpAct a = mlp_warp(w, x, sa[warp][0], sa[warp][1]);
  if (lane < MLP_OUT) coef[(size_t)MLP_OUT * s + lane] = (double)a.c;
}

// training, part 1: per sample (warp) forward, loss, and the back-propagated
// signals dc (9), d2 (64), d1 (64) plus the activations needed for the weight
// gradients; the loss of each sample goes to loss[b].
__global__ void __launch_bounds__(256) k_mlp_train_fwd(const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ feat, const float* __restrict__ G,
                                                       const float* __restrict__ h, const int* __restrict__ idx, int B,
                                                       float* __restrict__ sx, float* __restrict__ sa1,
                                                       float* __restrict__ sa2, float* __restrict__ sd1,
                                                       float* __restrict__ sd2, float* __restrict__ sdc,
                                                       float* __restrict__ loss, float rel_err) {
  __shared__ float sa[8][4][MLP_H];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + warp;
  if (b >= B) return;
  const int s = idx[b];
  float x[MLP_IN];
  load_features(feat + (size_t)MLP_IN * s, x);
  float* a1 = sa[warp][0];
  float* a2 = sa[warp][1];
  float* d2s = sa[warp][2];
  MlpAct a = mlp_warp(w, x, a1, a2);
  // dL/dc = 2 (G c - h) / B, L = 1 - 2 c.h + c.G c; with rel_err > 0 the
  // objective adds e (2 |c|.|h| + |c|.|G| |c|) (G symmetric), whose
  // derivative is 2 e sgn(c) (|h| + |G| |c|)
  const float* Gs = G + (size_t)81 * s;
  const float* hs = h + (size_t)9 * s;
  float gc = 0.f, agc = 0.f, dc = 0.f, lterm = 0.f;
#pragma unroll
  for (int p = 0; p < MLP_OUT; ++p) {
    const float cp = __shfl_sync(0xffffffffu, a.c, p);
    if (lane < MLP_OUT) {
      gc = fmaf(Gs[lane * 9 + p], cp, gc);
      agc = fmaf(fabsf(Gs[lane * 9 + p]), fabsf(cp), agc);
    }
  }
  if (lane < MLP_OUT) {
    dc = 2.f * (gc - hs[lane]) / (float)B;
    lterm = a.c * gc - 2.f * a.c * hs[lane];
    if (rel_err > 0.f) {
      const float ac = fabsf(a.c), ah = fabsf(hs[lane]);
      const float sg = (float)((a.c > 0.f) - (a.c < 0.f));
      lterm = fmaf(rel_err, fmaf(2.f * ac, ah, ac * agc), lterm);
      dc = fmaf(2.f * rel_err * sg, (ah + agc) / (float)B, dc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lterm += __shfl_xor_sync(0xffffffffu, lterm, o);
  if (lane == 0) loss[b] = 1.f + lterm;
  // d2_k = (sum_o W3[o][k] dc_o) * (z2_k > 0)
  float dcv[MLP_OUT];
#pragma unroll
  for (int o = 0; o < MLP_OUT; ++o) dcv[o] = __shfl_sync(0xffffffffu, dc, o);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = lane + 32 * q;
    float t = 0.f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) t = fmaf(wbf(w, OW3 + o * MLP_H + k), dcv[o], t);
    const float d2 = a.z2[q] > 0.f ? t : 0.f;
    d2s[k] = d2;
    sd2[(size_t)MLP_H * b + k] = d2;
    sa1[(size_t)MLP_H * b + k] = a1[k];
    sa2[(size_t)MLP_H * b + k] = a2[k];
  }
  __syncwarp();
  // d1_j = (sum_k W2[k][j] d2_k) * (z1_j > 0)
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    float t = 0.f;
    for (int k = 0; k < MLP_H; ++k) t = fmaf(wbf(w, OW2 + k * MLP_H + j), d2s[k], t);
    sd1[(size_t)MLP_H * b + j] = a.z1[q] > 0.f ? t : 0.f;
  }
  if (lane < MLP_IN) sx[(size_t)MLP_IN * b + lane] = x[lane];
  if (lane < MLP_OUT) sdc[(size_t)MLP_OUT * b + lane] = dc;
}

// training, part 2: one thread per parameter sums its gradient over the batch
// in a fixed order (deterministic), then (apply != 0) takes one Adam step on
// the FP32 master weight and refreshes the bfloat16 copy.
__global__ void __launch_bounds__(256) k_mlp_train_grad(float* __restrict__ w32, __nv_bfloat16* __restrict__ w16,
                                                        float* __restrict__ m, float* __restrict__ v, int B,
                                                        const float* __restrict__ sx, const float* __restrict__ sa1,
                                                        const float* __restrict__ sa2, const float* __restrict__ sd1,
                                                        const float* __restrict__ sd2, const float* __restrict__ sdc,
                                                        double* __restrict__ grad_out, int apply, int t, float lr,
                                                        float beta1, float beta2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  // gradient = sum_b left[b][i] * right[b][j] for the parameter's (i, j)
  const float *L, *Rr;
  int ls, rs, li, rj;
  if (p < OB1) { L = sd1; ls = MLP_H; li = p / MLP_IN; Rr = sx; rs = MLP_IN; rj = p % MLP_IN; }
  else if (p < OW2) { L = sd1; ls = MLP_H; li = p - OB1; Rr = nullptr; rs = 0; rj = 0; }
  else if (p < OB2) { const int q = p - OW2; L = sd2; ls = MLP_H; li = q / MLP_H; Rr = sa1; rs = MLP_H; rj = q % MLP_H; }
  else if (p < OW3) { L = sd2; ls = MLP_H; li = p - OB2; Rr = nullptr; rs = 0; rj = 0; }
  else if (p < OB3) { const int q = p - OW3; L = sdc; ls = MLP_OUT; li = q / MLP_H; Rr = sa2; rs = MLP_H; rj = q % MLP_H; }
  else { L = sdc; ls = MLP_OUT; li = p - OB3; Rr = nullptr; rs = 0; rj = 0; }
  double g = 0.0;
  for (int b = 0; b < B; ++b) {
    const float l = L[(size_t)ls * b + li];
    g += Rr ? (double)l * (double)Rr[(size_t)rs * b + rj] : (double)l;
  }
  if (grad_out) grad_out[p] = g;
  if (!apply) return;
  const float gf = (float)g;
  const float mm = beta1 * m[p] + (1.f - beta1) * gf;
  const float vv = beta2 * v[p] + (1.f - beta2) * gf * gf;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(beta1, (float)t));
  const float vh = vv / (1.f - powf(beta2, (float)t));
  const float nw = w32[p] - lr * mh / (sqrtf(vh) + eps);
  w32[p] = nw;
  w16[p] = __float2bfloat16_rn(nw);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

void launch_mlp_forward(const __nv_bfloat16* w, const float* feat, int S, double* coef, cudaStream_t st) {
  if (S > 0) k_mlp_forward<<<(S + 7) / 8, 256, 0, st>>>(w, feat, S, coef);
}
void launch_mlp_train(const MlpTrainArgs& a, cudaStream_t st) {
  k_mlp_train_fwd<<<(a.B + 7) / 8, 256, 0, st>>>(a.w16, a.feat, a.G, a.h, a.idx, a.B, a.sx, a.sa1, a.sa2, a.sd1,
                                                 a.sd2, a.sdc, a.loss, a.rel_err);
  k_mlp_train_grad<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(a.w32, a.w16, a.m, a.v, a.B, a.sx, a.sa1, a.sa2,
                                                             a.sd1, a.sd2, a.sdc, a.grad_out, a.apply, a.t, a.lr,
                                                             a.beta1, a.beta2, a.eps);
}
void launch_to_bf16(const float* a, __nv_bfloat16* b, int n, cudaStream_t st) {
  k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(a, b, n);
}

// ---------------------------------------------------------------- features per system
// raw features of each system for the current step: (dt, q_s * |fq|, D, kappa, h)
__global__ void k_features(const double* __restrict__ q, int R, double dt, double fq, double D, double kap, double hh,
                           float* __restrict__ feat) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= R) return;
  float* f = feat + (size_t)MLP_IN * s;
  f[0] = (float)dt;
  f[1] = (float)(q[s] * fabs(fq));
  f[2] = (float)D;
  f[3] = (float)kap;
  f[4] = (float)hh;
}
void launch_features(const double* q, int R, double dt, double fq, double D, double kap, double hh, float* feat,
                     cudaStream_t st) {
  k_features<<<(R + 255) / 256, 256, 0, st>>>(q, R, dt, fq, D, kap, hh, feat);
}

// ---------------------------------------------------------------- Horner SpMM
// z_out = D^-1 (c_j r + L z_in) for systems in polynomial mode (pmode[s] = 1),
// with c_j = coef[s][j] (cj_index j); FIRST: z_out = c_8 D^-1 r (no SpMM) for
// polynomial systems and D^-1 r for Jacobi systems.  Lane mapping and layout
// as in k_spmm.cu.
template <int NB, bool TRANSF>
__global__ void __launch_bounds__(256) k_spmm_horner(OpArgs op, VecArgs va, const float2* __restrict__ zin,
                                                     const float2* __restrict__ r, float2* __restrict__ zout,
                                                     const double* __restrict__ coef, int j,
                                                     const int* __restrict__ active, const int* __restrict__ pmode,
                                                     const int* __restrict__ n_active) {
  if (*n_active == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int r0 = (blockIdx.y * 32 + lane) * NB;
  const int c0 = blockIdx.y * 32 * NB + lane;
  const bool on = r0 < op.R;
  LaneCoef<NB> lc;
  lane_coef<NB>(op, 0, on ? r0 : 0, active, lc);
  bool any = false;
  float cj[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int s = r0 + b;
    const bool poly = on && lc.act[b] && pmode[s];
    any |= poly;
    cj[b] = poly ? (float)coef[(size_t)MLP_OUT * s + j] : 0.f;
  }
  if (!__any_sync(0xffffffffu, any)) return;
  const float qx = (float)lc.qx, qy = (float)lc.qy, qz = (float)lc.qz, ca = (float)lc.a;
  BT_FOR_CHUNKED_ROWS(row, op.n, warp, W) {
    const int k0 = op.rp[row], k1 = op.rp[row + 1];
    float2 P[NB], Q[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) P[b] = Q[b] = make_float2(0.f, 0.f);
    for (int k = k0; k < k1; ++k) {
      const int jc = __ldg(op.col + k);
      const float4 v = __ldg(op.pk32 + k);
      const float m = qx * v.y + qy * v.z + qz * v.w;
      float z1 = 0.f;
      if constexpr (TRANSF) z1 = __ldg(op.p1_32 + k);
      if (!on) continue;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const float2 xv = __ldg(zin + (size_t)jc * op.Rp + c0 + 32 * b);
        float c = ca * v.x;
        if constexpr (TRANSF) c = fmaf((float)lc.b[b], z1, c);
        P[b].x = fmaf(c, xv.x, P[b].x);
        P[b].y = fmaf(c, xv.y, P[b].y);
        Q[b].x = fmaf(m, xv.x, Q[b].x);
        Q[b].y = fmaf(m, xv.y, Q[b].y);
      }
    }
    if (!on) continue;
    const float4 dg = va.diag32[row];
    const float dmd = TRANSF ? va.diag_md32[row] : 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int s = r0 + b;
      if (!(lc.act[b] && pmode[s])) continue;
      const size_t e = (size_t)row * op.Rp + c0 + 32 * b;
      const float cc = (float)lc.c[b];
      float2 y = make_float2(P[b].x - cc * Q[b].y, P[b].y + cc * Q[b].x);
      const float2 rv = r[e];
      y.x = fmaf(cj[b], rv.x, y.x);
      y.y = fmaf(cj[b], rv.y, y.y);
      float dre = dg.x;
      if constexpr (TRANSF) dre = fmaf((float)lc.b[b], dmd, dre);
      const float dim = cc * (qx * dg.y + qy * dg.z + qz * dg.w);
      const float den = 1.f / (dre * dre + dim * dim);
      zout[e] = make_float2((y.x * dre + y.y * dim) * den, (y.y * dre - y.x * dim) * den);
    }
  }
}

// z = c_8 D^-1 r (polynomial systems) or D^-1 r (Jacobi systems), elementwise
__global__ void k_horner_first(OpArgs op, VecArgs va, const float2* __restrict__ r, float2* __restrict__ z,
                               const double* __restrict__ coef, const int* __restrict__ active,
                               const int* __restrict__ pmode, const int* __restrict__ n_active) {
  if (*n_active == 0) return;
  const size_t N = (size_t)va.n * va.Rp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(e % va.Rp);
    const int s = sys_of_col(col, va.nb);
    if (s >= va.R || !active[s]) continue;
    const int64_t i = (int64_t)(e / va.Rp);
    const OpCoef cf = op_coef(op, 0);
    const double q = op.q[s];
    const float bb = (float)(cf.bq2 * q * q), cc = (float)(cf.cq * q);
    const float4 dg = va.diag32[i];
    float dre = dg.x;
    if (op.transformed) dre = fmaf(bb, va.diag_md32[i], dre);
    const float dim = cc * ((float)op.qhat[3 * s] * dg.y + (float)op.qhat[3 * s + 1] * dg.z +
                            (float)op.qhat[3 * s + 2] * dg.w);
    const float c8 = pmode[s] ? (float)coef[(size_t)MLP_OUT * s + 8] : 1.f;
    const float2 rv = r[e];
    const float den = c8 / (dre * dre + dim * dim);
    z[e] = make_float2((rv.x * dre + rv.y * dim) * den, (rv.y * dre - rv.x * dim) * den);
  }
}

// rho = <r, z> (unconjugated for COCG, conjugated for CG) for the
// polynomial-preconditioned update; last block forms beta and the
// convergence bookkeeping exactly as k_krylov_update does for Jacobi.
template <bool CONJ>
__global__ void __launch_bounds__(256) k_precond_dot(VecArgs va, const float2* __restrict__ r,
                                                     const float2* __restrict__ z, KrylovState ks, RedScratch rs,
                                                     int* __restrict__ pmode, int init) {
  if (*ks.n_active == 0) return;
  __shared__ double2 sm[256];
  const int t = threadIdx.x;
  // one system column per thread slot, rows strided (as the element kernels)
  const int RS = va.Rp < 256 ? va.Rp : 256, rpp = 256 / RS;
  double2 acc[4];
  for (int k = 0; k < 4; ++k) acc[k] = make_double2(0, 0);
  const int64_t per = (va.n + gridDim.x - 1) / gridDim.x;
  const int64_t rb = (int64_t)blockIdx.x * per, re = min(va.n, rb + per);
  if (t < rpp * RS) {
    const int rr = t % RS, ro = t / RS;
    for (int k = 0; k < (va.Rp + 255) / 256 && k < 4; ++k) {
      const int col = rr + 256 * k;
      if (col >= va.Rp) continue;
      const int s = sys_of_col(col, va.nb);
      if (s >= va.R || !ks.active[s] || !pmode[s]) continue;
      float2 a = make_float2(0.f, 0.f);
      int cnt = 0;
      for (int64_t i = rb + ro; i < re; i += rpp) {
        const size_t e = (size_t)i * va.Rp + col;
        float2 rv = r[e];
        const float2 zv = z[e];
        if (CONJ) rv.y = -rv.y;
        a.x += rv.x * zv.x - rv.y * zv.y;
        a.y += rv.x * zv.y + rv.y * zv.x;
        if (++cnt == 32) {
          cnt = 0;
          acc[k].x += a.x;
          acc[k].y += a.y;
          a = make_float2(0.f, 0.f);
        }
      }
      acc[k].x += a.x;
      acc[k].y += a.y;
    }
  }
  // block partials at the logical system index
  if ((va.Rp + 255) / 256 == 1) {
    sm[t] = acc[0];
    __syncthreads();
    if (t < RS) {
      double2 s2 = make_double2(0, 0);
      for (int o = 0; o < rpp; ++o) {
        s2.x += sm[o * RS + t].x;
        s2.y += sm[o * RS + t].y;
      }
      reinterpret_cast<double2*>(rs.part)[(size_t)blockIdx.x * va.Rp + sys_of_col(t, va.nb)] = s2;
    }
  } else {
    for (int k = 0; k < 4; ++k) {
      const int col = t + 256 * k;
      if (col < va.Rp) reinterpret_cast<double2*>(rs.part)[(size_t)blockIdx.x * va.Rp + sys_of_col(col, va.nb)] = acc[k];
    }
  }
  if (!last_block(rs.counter, gridDim.x)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < va.R; s += blockDim.x) {
    if (!ks.active[s]) continue;
    if (!pmode[s]) {  // Jacobi system: its rho and beta came from the update kernel
      if (init) {     // (at a solve's start: p = D^-1 r, beta = 0)
        ks.beta[2 * s] = 0;
        ks.beta[2 * s + 1] = 0;
      }
      atomicAdd(&s_cnt, 1);
      continue;
    }
    double2 o = make_double2(0, 0);
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(rs.part) + (size_t)b * va.Rp + s);
      o.x += v.x;
      o.y += v.y;
    }
    const double2 rho = make_double2(ks.rho[2 * s], ks.rho[2 * s + 1]);
    const double den = rho.x * rho.x + rho.y * rho.y;
    // breakdown: rho = 0, or a preconditioner that is not positive on the
    // Hermitian (CG) system; hand the system back to Jacobi for the rest of the step
    const double on2 = o.x * o.x + o.y * o.y;
    if (!(init || den > 0) || !(on2 > 0) || !isfinite(o.x) || !isfinite(o.y) || (CONJ && !(o.x > 0))) {
      ks.active[s] = 0;
      pmode[s] = 0;
      continue;
    }
    if (init) {
      ks.beta[2 * s] = 0;
      ks.beta[2 * s + 1] = 0;
    } else {
      ks.beta[2 * s] = (o.x * rho.x + o.y * rho.y) / den;
      ks.beta[2 * s + 1] = (o.y * rho.x - o.x * rho.y) / den;
    }
    ks.rho[2 * s] = o.x;
    ks.rho[2 * s + 1] = o.y;
    atomicAdd(&s_cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

#define BT_DISPATCH_NB(nb, ...)                                 \
  switch (nb) {                                                 \
    case 4: { constexpr int NB_ = 4; __VA_ARGS__; } break;      \
    case 2: { constexpr int NB_ = 2; __VA_ARGS__; } break;      \
    default: { constexpr int NB_ = 1; __VA_ARGS__; } break;     \
  }

void launch_horner(const OpArgs& op, const VecArgs& va, const float2* zin, const float2* r, float2* zout,
                   const double* coef, int j, const int* active, const int* pmode, const int* n_active, int sms,
                   cudaStream_t st) {
  if (j == MLP_OUT - 1) {
    k_horner_first<<<(unsigned)std::min<int64_t>(4096, ((int64_t)va.n * va.Rp + 255) / 256), 256, 0, st>>>(
        op, va, r, zout, coef, active, pmode, n_active);
    return;
  }
  BT_DISPATCH_NB(va.nb, {
    dim3 grid(spmm_grid_rows(op.n, sms), (op.R + 32 * NB_ - 1) / (32 * NB_));
    if (op.transformed) k_spmm_horner<NB_, true><<<grid, 256, 0, st>>>(op, va, zin, r, zout, coef, j, active, pmode, n_active);
    else k_spmm_horner<NB_, false><<<grid, 256, 0, st>>>(op, va, zin, r, zout, coef, j, active, pmode, n_active);
  })
}

void launch_precond_dot(const VecArgs& va, const float2* r, const float2* z, const KrylovState& ks, RedScratch rs,
                        int* pmode, int conj, int init, int sms, cudaStream_t st) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * REDUCE_BLOCKS_PER_SM, va.n));
  if (conj) k_precond_dot<true><<<g, 256, 0, st>>>(va, r, z, ks, rs, pmode, init);
  else k_precond_dot<false><<<g, 256, 0, st>>>(va, r, z, ks, rs, pmode, init);
}

// ---------------------------------------------------------------- Gram data for training
// V holds v_0..v_9 (10 vectors [n][Rp]); y_j = diag(L) v_{j+1}; per system:
// G_jk = Re(y_j^H y_k), h_j = Re(y_j^H r), and |r|^2, summed over rows.
constexpr int NGRAM = 45 + 9 + 1;
__global__ void __launch_bounds__(256) k_gram(OpArgs op, VecArgs va, const float2* __restrict__ r,
                                              const float2* __restrict__ V, size_t vstride,
                                              double* __restrict__ part, int nbx_total, unsigned int* counter,
                                              double* __restrict__ out) {
  // one thread per (row, system); block partials per system in part[block][s][NGRAM]
  const int RS = va.Rp < 256 ? va.Rp : 256, rpp = 256 / RS;
  const int t = threadIdx.x;
  float acc[NGRAM];
#pragma unroll
  for (int k = 0; k < NGRAM; ++k) acc[k] = 0.f;
  const int64_t per = (va.n + gridDim.x - 1) / gridDim.x;
  const int64_t rb = (int64_t)blockIdx.x * per, re = min(va.n, rb + per);
  const int col = (t % RS) + RS * blockIdx.y;
  const bool live = t < rpp * RS && col < va.Rp;
  const int s = live ? sys_of_col(col, va.nb) : 0;
  if (live && s < va.R) {
    const OpCoef cf = op_coef(op, 0);
    const double q = op.q[s];
    const float bb = (float)(cf.bq2 * q * q), cc = (float)(cf.cq * q);
    const float qx = (float)op.qhat[3 * s], qy = (float)op.qhat[3 * s + 1], qz = (float)op.qhat[3 * s + 2];
    for (int64_t i = rb + t / RS; i < re; i += rpp) {
      const size_t e = (size_t)i * va.Rp + col;
      const float4 dg = va.diag32[i];
      float dre = dg.x;
      if (op.transformed) dre = fmaf(bb, va.diag_md32[i], dre);
      const float dim = cc * (qx * dg.y + qy * dg.z + qz * dg.w);
      float2 y[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const float2 v = V[(size_t)(j + 1) * vstride + e];
        y[j] = make_float2(dre * v.x - dim * v.y, dre * v.y + dim * v.x);
      }
      const float2 rv = r[e];
      int k = 0;
#pragma unroll
      for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = a; b < 9; ++b) acc[k++] += y[a].x * y[b].x + y[a].y * y[b].y;
#pragma unroll
      for (int a = 0; a < 9; ++a) acc[45 + a] += y[a].x * rv.x + y[a].y * rv.y;
      acc[54] += rv.x * rv.x + rv.y * rv.y;
    }
  }
  // reduce threads of the same system inside the block (fixed order via smem)
  __shared__ float sm[256];
  for (int k = 0; k < NGRAM; ++k) {
    sm[t] = acc[k];
    __syncthreads();
    if (t < RS) {
      double a = 0;
      for (int o = 0; o < rpp; ++o) a += sm[o * RS + t];
      const int c = t + RS * blockIdx.y;
      if (c < va.Rp) part[((size_t)blockIdx.x * va.Rp + sys_of_col(c, va.nb)) * NGRAM + k] = a;
    }
    __syncthreads();
  }
  if (!last_block(counter, gridDim.x * gridDim.y)) return;
  for (int w = threadIdx.x; w < va.R * NGRAM; w += blockDim.x) {
    const int ss = w / NGRAM, k = w % NGRAM;
    double a = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) a += __ldcg(part + ((size_t)b * va.Rp + ss) * NGRAM + k);
    out[(size_t)ss * NGRAM + k] = a;
  }
}

void launch_gram(const OpArgs& op, const VecArgs& va, const float2* r, const float2* V, size_t vstride,
                 double* part, unsigned int* counter, double* out, int sms, cudaStream_t st) {
  const int RS = va.Rp < 256 ? va.Rp : 256;
  dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 2, va.n)), (va.Rp + RS - 1) / RS);
  k_gram<<<grid, 256, 0, st>>>(op, va, r, V, vstride, part, grid.x * grid.y, counter, out);
}

}  // namespace bt
