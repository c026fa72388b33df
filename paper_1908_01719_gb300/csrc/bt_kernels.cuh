// Kernel argument structures, device helpers and launch wrappers of libbtgpu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "bt_internal.h"

namespace bt {

// ---------------------------------------------------------------- assembly
struct AsmArgs {
  const double* xyz;
  const int32_t* tets;
  const int32_t* cmpt;
  const double* Dc;
  const double* invT2c;  // [n_cmpt] 1/T2 per compartment (or null: none)
  const double* Dten;    // [n_cmpt][6] diffusion tensors (or null: isotropic Dc)
  const double* DtenE;   // [n_elem][6] per-element tensors, overriding Dten (or null)
  double centre[3];
  int64_t nt, nf, nnz;
  int nv;       // 4 tetrahedra, 3 triangles, 2 segments
  int surface;  // triangles of a surface in 3-D (else in the xy plane)
  const int32_t* face_ta;
  const int8_t* face_lv;
  const double* face_kappa;
  const int64_t* tc_ptr;
  const int32_t* tc;
  const int64_t* fc_ptr;
  const int32_t* fc;
  double* geo;     // 33 nt
  double* fcoef;   // nf
  double* planes;  // 11 nnz
};
void launch_assembly(const AsmArgs& a, cudaStream_t st);

struct DeriveArgs {
  const double* planes;
  int64_t nnz, n;
  double thdt;
  int transformed;
  const int32_t* rp;
  const int32_t* col;
  double* A0;
  double* KJ;
  double4* pk64;
  float4* pk32;
  float* md32;
  float4* pkhi;
  float4* pklo;
  float2* kjmd_hi;
  float2* kjmd_lo;
  double* w;
  double4* diag64;
  double* diag_md64;
  float4* diag32;
  float* diag_md32;
  const double* MB;  // [nnz] kappa_e x boundary-face mass (weak periodic box) or null
  double theta;
};
void launch_derive(const DeriveArgs& a, cudaStream_t st);

// ---------------------------------------------------------------- solver state
// Per-system (right-hand side) Krylov scalars, FP64.
struct KrylovState {
  double* rho;       // complex rho: [2 * n_sys] (COCG scalars are complex)
  double* alpha;     // complex alpha: [2 * n_sys]
  double* beta;      // complex beta:  [2 * n_sys]
  double* rr0;       // |r_0|^2 of the current solve
  double* rr;        // |r|^2
  double* tol2;      // stop when rr <= tol2
  int* iter;
  int* active;
  int* n_active;     // device counter of active systems
  int* status;       // BT_OK / BT_ENOCONV / BT_ENAN per system
  double* rr_best;   // smallest |r|^2 seen in the current solve
  int* it_best;      // iteration at which it was seen
  int max_iter;
  int stall;         // > 0: stop a solve after `stall` iterations without a new best
  // halo-tile iteration only (null otherwise)
  int* par;          // device: which of the two p buffers holds the current p
  int* pend;         // per system: x += alpha p of the last apply still to do
  unsigned long long* sys_iter;  // device [1 + G]: active systems summed over SpMM launches, in all
                                 // and per segment (or null)
};

// Per-system refinement scalars.
struct RefineState {
  double* r0n2;      // |r_0|^2 of the step
  double* rk2;       // |r_k|^2
  double* scale;     // |r_k| used to normalise the inner right-hand side
  double* err;       // accumulated |r_final| / |r_0|
  int* active;
  int* n_active;
  double tol2;       // tol_ref^2
  double floor_c2;   // (eps * max w)^2: |r_0|^2 below floor_c2 |u|^2 counts as zero
  int* status;       // per-system status (shared with the Krylov state)
};

// Segment plan: the solve may hold several geometries ("segments") of uneven
// size as one block-diagonal system.  Segment g owns rows [row0[g], row0[g+1])
// and systems [g R, (g+1) R); every block of a launch works inside one
// segment (blocks blk0[g] .. blk0[g+1]-1), so block partial sums never mix
// geometries.
struct SegPlan {
  const int* blk_seg;   // [nblk] segment of each block
  const int* blk0;      // [G+1] first block of each segment
  const int64_t* row0;  // [G+1] first row of each segment
  int G;
  int nblk;
};

// Operator description shared by all fused SpMM kernels.
//   y_r = a (P0 x_r) + bq2 q_r^2 (P1 x_r) + i cq q_r (qhat_d . Pd) x_r
struct OpArgs {
  const int32_t* rp;
  const int32_t* col;
  int64_t n;
  const double4* pk64;   // {A0, d0, d1, d2}
  const double* p0_64;   // P0 override (K + J), or null: P0 = A0
  const double* p1_64;   // D-weighted mass (transformed frame) or null
  const float4* pk32;
  const float* p1_32;
  const float4* pkhi;    // double-float split of pk64
  const float4* pklo;
  const float2* kjmd_hi; // double-float split of (K + J, MD)
  const float2* kjmd_lo;
  const OpCoef* coef;    // device: one per segment for the current step, or (step != null)
                         // the whole table [step][2][segment]
  const int* step;       // device step counter (captured time step) or null
  int sel;               // with step: 0 = r_0 operator, 1 = L_n
  const double* q;       // [G R]
  const double* qhat;    // [3 G R] unit direction of each system
  int R, Rp;             // systems per segment, padded vector width
  int transformed;
  SegPlan sp;
};

// Halo tiles of the shared-memory Krylov apply (HaloTiles on the device).
struct HaloArgs {
  const int32_t* t_r0;      // [ntiles + 1] offsets into rows
  const int32_t* rows;      // owned rows, tile by tile
  const int32_t* rowe;      // [n + 1] first entry of each owned row (tile order)
  const uint16_t* rowl;     // local halo index of each owned row
  const int32_t* u0;        // [ntiles + 1] offsets into ucol
  const int32_t* e0;        // [ntiles + 1] first entry of each tile
  const uint32_t* ucol;     // halo rows, bit 31 = owned
  const uint16_t* lidx;     // [nnz] local column index of each entry
  const float4* pkt;        // [nnz] {A0, d0, d1, d2} in tile-entry order
  const float* mdt;         // [nnz] MD in tile-entry order
  const float4* dft;        // [3 nnz] double-float planes in tile-entry order
  const int32_t* seg_tile0; // [G + 1]
  int umax;
};

struct VecArgs {
  int64_t n;
  int R, Rp, nb;
  SegPlan sp;
  const double4* diag64;
  const double* diag_md64;
  const float4* diag32;
  const float* diag_md32;
};

// Weak pseudo-periodic coupling rows on the device (WeakPeriodic).
struct WeakArgs {
  const int32_t* rows;
  const int32_t* ptr;
  const int32_t* col;
  const double* w;
  const int8_t* code;
  int64_t nr;
  double L[3];
  double scale;         // theta dt kappa_e
  const double* F;      // [N + 1] F(t_n)
  const int* step_dev;  // captured step counter, or null
  int step_host;
};

// partial-sum scratch for the deterministic last-block reductions
struct RedScratch {
  double* part;          // [max_blocks * Rp * 4]
  unsigned int* counter; // one per reduction site
};

// learned polynomial preconditioner (k_precond.cu)
constexpr int MLP_IN = 5, MLP_H = 64, MLP_OUT = 9;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
struct MlpTrainArgs {
  float* w32;
  __nv_bfloat16* w16;
  float *m, *v;
  const float *feat, *G, *h;
  const int* idx;
  int B;
  float *sx, *sa1, *sa2, *sd1, *sd2, *sdc, *loss;
  double* grad_out;
  int apply, t;
  float lr, beta1, beta2, eps;
  // > 0: the objective adds the loss's spread for data known to this
  // relative accuracy, rel_err (2 |c|.|h| + |c|.|G| |c|) per sample
  float rel_err;
};
void launch_mlp_forward(const __nv_bfloat16* w, const float* feat, int S, double* coef, cudaStream_t st);
void launch_mlp_train(const MlpTrainArgs& a, cudaStream_t st);
void launch_to_bf16(const float* a, __nv_bfloat16* b, int n, cudaStream_t st);
void launch_features(const double* q, int R, double dt, double fq, double D, double kap, double hh, float* feat,
                     cudaStream_t st);

// launch wrappers (k_spmm.cu / k_krylov.cu)
enum { REDUCE_BLOCKS_PER_SM = 4 };
int spmm_grid_rows(int64_t n, int sms);

void launch_spmm_krylov_f32(const OpArgs& op, const float2* p, float2* q, const KrylovState& ks,
                            RedScratch rs, int conj, int nb, int sms, cudaStream_t st);
void launch_gather_tile_planes(const int32_t* slot, int64_t nnz, const float4* pk32, const float* md32, float4* pkt,
                               float* mdt, cudaStream_t st);
void launch_spmm_krylov_f64(const OpArgs& op, const double2* p, double2* q, const KrylovState& ks,
                            RedScratch rs, int conj, int nb, int sms, cudaStream_t st);
// r = op_{P0=K+J}(u) with |r|^2, |u|^2 partials; sets refinement state
void launch_resid0(const OpArgs& op, const double2* u, double2* r, const RefineState& rf, RedScratch rs,
                   int nb, int sms, cudaStream_t st);
// u += s d; r -= s op_{P0=A0}(d) with |r|^2 partials; updates refinement state
void launch_resid_sub(const OpArgs& op, const float2* d, double2* u, double2* r, const RefineState& rf,
                      RedScratch rs, int nb, int sms, cudaStream_t st);
// the same two residual kernels in double-float arithmetic (u, r stored as
// {re_hi, im_hi, re_lo, im_lo} FP32 quadruples)
void launch_resid0_df(const OpArgs& op, const float4* u, float4* r, const RefineState& rf, RedScratch rs,
                      int nb, int sms, cudaStream_t st);
void launch_resid_sub_df(const OpArgs& op, const float2* d, float4* u, float4* r, const RefineState& rf,
                         RedScratch rs, int nb, int sms, cudaStream_t st);
// the same over the halo tiles (the halo-staged variant)
void resid_df_halo_prepare();
void launch_gather_tile_df(const int32_t* slot, int64_t nnz, const float4* pkhi, const float4* pklo, const float2* kh,
                           const float2* kl, float4* out, cudaStream_t st);
bool resid_df_halo_available(int nb, int mode);
void launch_resid0_df_halo(const OpArgs& op, const HaloArgs& h, const float4* u, float4* r, const RefineState& rf,
                           RedScratch rs, int nb, cudaStream_t st);
void launch_resid_sub_df_halo(const OpArgs& op, const HaloArgs& h, const float2* d, float4* u, float4* r,
                              const RefineState& rf, RedScratch rs, int nb, cudaStream_t st);
void launch_krylov_init_f32_df(const OpArgs& op, const VecArgs& va, const float4* rdf, const double* scale,
                               const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks,
                               double tol, RedScratch rs, int conj, int sms, cudaStream_t st);
void launch_signal_df(const VecArgs& va, const double* w, const float4* u, double* S, RedScratch rs, int sms,
                      cudaStream_t st);
void launch_fill_u_df(const VecArgs& va, float4* u, const double* rho, cudaStream_t st);

void launch_spmm_krylov_f64_narrow(const OpArgs& op, const double2* p, double2* q, const KrylovState& ks,
                                   RedScratch rs, int conj, int sms, cudaStream_t st);
void launch_resid0_narrow(const OpArgs& op, const double2* u, double2* r, const RefineState& rf, RedScratch rs,
                          int sms, cudaStream_t st);
void launch_krylov_init_f32(const OpArgs& op, const VecArgs& va, const double2* r64, const double* scale,
                            const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks,
                            double tol, RedScratch rs, int conj, int sms, cudaStream_t st);
void launch_krylov_update_f32(const OpArgs& op, const VecArgs& va, float2* x, float2* r, const float2* p,
                              const float2* q, const KrylovState& ks, RedScratch rs, int conj, int sms,
                              cudaStream_t st, int* pmode = nullptr);
void launch_krylov_p_f32(const OpArgs& op, const VecArgs& va, const float2* r, float2* p, const KrylovState& ks,
                         int sms, cudaStream_t st, const float2* zbuf = nullptr, const int* pmode = nullptr);
// polynomial preconditioner application and its inner product
void launch_horner(const OpArgs& op, const VecArgs& va, const float2* zin, const float2* r, float2* zout,
                   const double* coef, int j, const int* active, const int* pmode, const int* n_active, int sms,
                   cudaStream_t st);
void launch_precond_dot(const VecArgs& va, const float2* r, const float2* z, const KrylovState& ks, RedScratch rs,
                        int* pmode, int conj, int init, int sms, cudaStream_t st);
void launch_gram(const OpArgs& op, const VecArgs& va, const float2* r, const float2* V, size_t vstride,
                 double* part, unsigned int* counter, double* out, int sms, cudaStream_t st);

// Halo-tile Jacobi iteration (FP32): the Krylov state keeps z = D^-1 r
// instead of r, and p in two buffers.  One iteration is
//   apply:  p = z + beta p_prev (halo rows staged in shared memory), deferred
//           x += alpha_prev p_prev, q = L p, alpha = rho / <p, q>
//   update: r = D z - alpha q, z = D^-1 r, rho' = <r, z>, |r|^2, beta
// and flush_x applies the last deferred x update after the loop.
void halo_prepare();
size_t halo_smem_bytes(int nb, int umax);
int halo_umax(int nb);  // halo rows per tile for a vector layout of nb columns per lane
void launch_spmm_halo(const OpArgs& op, const HaloArgs& h, const float2* z, float2* pA, float2* pB, float2* x,
                      float2* q, const KrylovState& ks, RedScratch rs, int conj, int nb, cudaStream_t st);
void launch_krylov_init_z(const OpArgs& op, const VecArgs& va, const void* rres, int df, const double* scale,
                          const int* ref_active, float2* x, float2* z, const KrylovState& ks, double tol,
                          RedScratch rs, int conj, cudaStream_t st);
void launch_krylov_update_z(const OpArgs& op, const VecArgs& va, float2* z, const float2* q, const KrylovState& ks,
                            RedScratch rs, int conj, cudaStream_t st);
void launch_flush_x(const VecArgs& va, float2* x, const float2* pA, const float2* pB, const KrylovState& ks,
                    cudaStream_t st);

// Slice-tiled Jacobi iteration (FP32, k_spmm_slice.cu): the vectors and the
// initialisation of the row variant (x, r, p, q), three launches per iteration:
//   spmm:   q = L p over 32-system slices of Morton tiles staged in shared
//           memory, (p, q); last block: alpha, pend = active
//   r:      r -= alpha q, rho' = (r, D^-1 r), |r|^2; last block: convergence
//           tests and beta
//   xp:     x += alpha p (pending systems), p = D^-1 r + beta p (active ones);
//           last block clears pend
// spt is the plan of tile blocks (each block of the SpMM launch is one tile
// block times one slice of 32 systems); the vector width Rp must be a
// multiple of 32 (and of 32 NB).
// cfg: the configuration (SLICE_CONF: tile class, stages, threads, blocks per
// SM); h must hold the tiles of that configuration's class.
void slice_prepare();
size_t slice_smem_bytes(int cfg);
void launch_spmm_slice(const OpArgs& op, const HaloArgs& h, const SegPlan& spt, const float2* p, float2* q,
                       const KrylovState& ks, RedScratch rs, int conj, int nb, int cfg, cudaStream_t st);
void launch_slice_r(const OpArgs& op, const VecArgs& va, float2* r, const float2* q, const KrylovState& ks,
                    RedScratch rs, int conj, cudaStream_t st);
void launch_slice_xp(const OpArgs& op, const VecArgs& va, float2* x, float2* p, const float2* r,
                     const KrylovState& ks, RedScratch rs, cudaStream_t st);
// start of an inner solve for the slice iteration (vectorised form of the row
// variant's initialisation): rres = the refinement residual (FP64 or, with df,
// double-float), r = rres / scale, p = D^-1 r, x = 0, rho, |r|^2
void launch_slice_init(const OpArgs& op, const VecArgs& va, const void* rres, int df, const double* scale,
                       const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks, double tol,
                       RedScratch rs, int conj, cudaStream_t st);

void launch_krylov_init_f64(const OpArgs& op, const VecArgs& va, const double2* r64, const int* ref_active,
                            double2* x, double2* r, double2* p, const KrylovState& ks, double tol, RedScratch rs,
                            int conj, int sms, cudaStream_t st);
void launch_krylov_update_f64(const OpArgs& op, const VecArgs& va, double2* x, double2* r, const double2* p,
                              const double2* q, const KrylovState& ks, RedScratch rs, int conj, int sms,
                              cudaStream_t st);
void launch_krylov_p_f64(const OpArgs& op, const VecArgs& va, const double2* r, double2* p,
                         const KrylovState& ks, int sms, cudaStream_t st);

void launch_axpy_u(const VecArgs& va, const double2* d, double2* u, const KrylovState& ks,
                   const RefineState& rf, int sms, cudaStream_t st);
void launch_fill_u(const VecArgs& va, double2* u, const double* rho, cudaStream_t st);
// r_0 += theta dt kappa_e C_n u (partner faces) and the step-start
// refinement bookkeeping redone on the new r_0 (weak pseudo-periodic box)
void launch_weak_coupling(const WeakArgs& wa, const VecArgs& va, const OpArgs& op, const void* u, void* r, int df,
                          cudaStream_t st);
void launch_resid0_renorm(const VecArgs& va, const void* u, const void* r, const RefineState& rf, RedScratch rs,
                          int df, cudaStream_t st);
void launch_extract_state(const void* u, int df, int64_t row0, int64_t rows, int Rp, int col, double2* out,
                          int sms, cudaStream_t st);
void launch_signal(const VecArgs& va, const double* w, const double2* u, double* S, RedScratch rs, int sms,
                   cudaStream_t st);
void launch_set_int(int* p, int v, int n, cudaStream_t st);
void launch_finish_step(const RefineState& rf, const KrylovState& ks, int R, cudaStream_t st);
void launch_mark_ref_left(const RefineState& rf, const KrylovState& ks, int R, cudaStream_t st);
void launch_seg_active(int* act, int R, int G, int step, const int* segN, cudaStream_t st);
// captured time step (k_graph.cu)
struct GraphCtl {
  int* ctl;        // [0] step, [1] refinement pass, [2] inner iteration, [3] total iterations, [4] total passes
  int* n_active;   // [0] Krylov, [1] refinement
  const int* segN;
  int R, G, max_iter, max_refine;
  int n_steps;     // time steps of the run (the outer WHILE node's bound)
};
void launch_graph_step_begin(const GraphCtl& c, int* rf_active, cudaStream_t st);
void launch_graph_cond(const GraphCtl& c, int which, cudaGraphConditionalHandle h, cudaStream_t st);
void launch_graph_step_end(const GraphCtl& c, cudaStream_t st);

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// 1/(a + ib)
__device__ __forceinline__ double2 crcp(double a, double b) {
  double d = 1.0 / (a * a + b * b);
  return make_double2(a * d, -b * d);
}
__device__ __forceinline__ float2 crcpf(float a, float b) {
  float d = 1.0f / (a * a + b * b);
  return make_float2(a * d, -b * d);
}

// Vector layout.  X is [n][Rp] complex; within each tile of 32*NB columns the
// column of system (RHS) s = tile*32*NB + l*NB + b is tile*32*NB + b*32 + l, so
// that lane l of a warp owns the NB consecutive systems of one direction and
// each of its NB loads is one contiguous 32-lane access.  NB = 1 is the
// identity.
__host__ __device__ __forceinline__ int sys_of_col(int c, int nb) {
  if (nb == 1) return c;
  const int t = c / (32 * nb), w = c - t * 32 * nb;
  return t * 32 * nb + (w & 31) * nb + (w >> 5);
}
__host__ __device__ __forceinline__ int col_of_sys(int s, int nb) {
  if (nb == 1) return s;
  const int t = s / (32 * nb), w = s - t * 32 * nb;
  return t * 32 * nb + (w % nb) * 32 + w / nb;
}

// Row order of the gathering kernels: blocks take 32-row chunks round-robin,
// so at any moment all blocks work inside one window of about
// gridDim.x * 32 rows; the +-1 z-plane neighbours of that window stay
// resident in L2 and each row of X is fetched from HBM about once.
constexpr int ROW_CHUNK = 32;
#define BT_FOR_CHUNKED_ROWS(row, n, first, stride)                                               \
  for (int64_t ch_ = blockIdx.x; ch_ * ROW_CHUNK < (int64_t)(n); ch_ += gridDim.x)                \
    for (int64_t row = ch_ * ROW_CHUNK + (first), re_ = min((int64_t)(n), (ch_ + 1) * ROW_CHUNK); \
         row < re_; row += (stride))
// the same inside the block's segment (sg_ = segment, rows [sr0_, sr1_))
#define BT_SEG_BEGIN(sp)                                                                          \
  const int sg_ = (sp).blk_seg[blockIdx.x];                                                       \
  const int sk_ = blockIdx.x - (sp).blk0[sg_], snb_ = (sp).blk0[sg_ + 1] - (sp).blk0[sg_];        \
  const int64_t sr0_ = (sp).row0[sg_], sr1_ = (sp).row0[sg_ + 1];
#define BT_FOR_SEG_CHUNKED_ROWS(row, first, stride)                                               \
  for (int64_t ch_ = sk_; sr0_ + ch_ * ROW_CHUNK < sr1_; ch_ += snb_)                             \
    for (int64_t row = sr0_ + ch_ * ROW_CHUNK + (first), re_ = min(sr1_, sr0_ + (ch_ + 1) * ROW_CHUNK); \
         row < re_; row += (stride))

// read-only 32-byte / 16-byte plane loads
__device__ __forceinline__ double4 ldg4(const double4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// Last-block-done: every block stores its partials, then the block that
// arrives last (atomic ticket, no waiting) reduces them in a fixed order.
__device__ __forceinline__ bool last_block(unsigned int* counter, unsigned int nblocks) {
  __shared__ unsigned int s_ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
  __syncthreads();
  bool last = (s_ticket == nblocks - 1);
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
  }
  return last;
}
// the NB values of one lane: base points at column tile*32*NB + lane
template <int NB, class T2>
__device__ __forceinline__ void load_x(const T2* __restrict__ p, T2 (&x)[NB]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) x[b] = __ldg(p + 32 * b);
}

// per-lane constants of the operator
template <int NB>
struct LaneCoef {
  double qx, qy, qz;
  double b[NB], c[NB];
  double a;
  int act[NB];
};

// coefficients of segment g for the current step
__device__ __forceinline__ OpCoef op_coef(const OpArgs& op, int g) {
  if (op.step) return op.coef[((size_t)(*op.step - 1) * 2 + op.sel) * op.sp.G + g];
  return op.coef[g];
}

// r0: first local system of the lane in segment g (global system g R + r)
template <int NB>
__device__ __forceinline__ void lane_coef(const OpArgs& op, int g, int r0, const int* active, LaneCoef<NB>& lc) {
  const OpCoef cf = op_coef(op, g);
  const int base = g * op.R;
  lc.a = cf.a;
  // the NB RHS of a lane share one direction (the host picks NB accordingly)
  const int d = base + (r0 < op.R ? r0 : 0);
  lc.qx = op.qhat[3 * d];
  lc.qy = op.qhat[3 * d + 1];
  lc.qz = op.qhat[3 * d + 2];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    int r = r0 + b;
    double q = r < op.R ? op.q[base + r] : 0.0;
    lc.b[b] = cf.bq2 * q * q;
    lc.c[b] = cf.cq * q;
    lc.act[b] = (r < op.R) && (active == nullptr || active[base + r]);
  }
}

// Reduce per-lane complex partials of NB RHS over the warps of the block and
// write them to part[blockIdx.x][r] (2 doubles per r).
template <int NB>
__device__ __forceinline__ void block_partials(double2 (&acc)[NB], int r0, int Rp, double* part) {
  __shared__ double2 sm[8][32][NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
#pragma unroll
  for (int b = 0; b < NB; ++b) sm[warp][lane][b] = acc[b];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double2 s = make_double2(0, 0);
      for (int w = 0; w < W; ++w) {
        s.x += sm[w][lane][b].x;
        s.y += sm[w][lane][b].y;
      }
      int r = r0 + b;
      if (r < Rp) reinterpret_cast<double2*>(part)[(size_t)blockIdx.x * Rp + r] = s;
    }
  }
}

// Single-segment variant over nbx blocks (kernels with their own grid).
template <class F>
__device__ __forceinline__ void reduce_partials_flat(const double* part, int nbx, int Rp, int R, F&& fn) {
  for (int s = threadIdx.x; s < R; s += blockDim.x) {
    double2 t = make_double2(0, 0);
    for (int b = 0; b < nbx; ++b) {
      double2 v = __ldcg(reinterpret_cast<const double2*>(part) + (size_t)b * Rp + s);
      t.x += v.x;
      t.y += v.y;
    }
    fn(s, t);
  }
}

// Sum over blocks b0..b1-1 of the NC complex partials part[(b Rp + r) NC + c]
// by one warp: lane l adds blocks b0 + l, b0 + l + 32, ... in order, then a
// fixed xor tree combines the lanes (the same order on every run); every lane
// gets the sums.  A block-sized last-block reduction done by one thread per
// system serialises hundreds of L2 round trips; this spreads them over 32.
template <int NC>
__device__ __forceinline__ void warp_sum_part(const double* part, int b0, int b1, int Rp, int r,
                                              double2 (&out)[NC]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c] = make_double2(0, 0);
  for (int b = b0 + lane; b < b1; b += 32)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(part) + ((size_t)b * Rp + r) * NC + c);
      out[c].x += v.x;
      out[c].y += v.y;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      out[c].x += __shfl_xor_sync(0xffffffffu, out[c].x, o);
      out[c].y += __shfl_xor_sync(0xffffffffu, out[c].y, o);
    }
}

// The NC complex block partials part[(b Rp + r) NC + c] of every system
// s = g R + r of a launch's segments, summed over the segment's blocks b in a
// fixed order and handed to fn(s, sums) by one thread; skip(s) leaves a system
// out.  A system is summed by one thread when the segments have few blocks and
// by one warp (warp_sum_part) when they have many: whichever costs fewer
// dependent L2 round trips per thread (many systems with few blocks each, as
// in a batch of small geometries, favour threads; few systems with hundreds of
// blocks favour warps).  The choice is the same in the whole block, whose size
// must be a multiple of 32.
template <int NC, class Skip, class F>
__device__ __forceinline__ void reduce_systems(const double* part, const SegPlan& sp, int R, int Rp, Skip&& skip,
                                               F&& fn) {
  const int GR = sp.G * R, nb = (sp.nblk + sp.G - 1) / sp.G;  // blocks per segment, on average
  const int nt = (int)blockDim.x, nw = nt >> 5;
  const bool by_warp =
      (int64_t)((GR + nt - 1) / nt) * nb > (int64_t)((GR + nw - 1) / nw) * ((nb + 31) / 32 + 5);
  if (by_warp) {
    for (int s = (int)(threadIdx.x >> 5); s < GR; s += nw) {
      if (skip(s)) continue;
      const int g = s / R;
      double2 o[NC];
      warp_sum_part<NC>(part, sp.blk0[g], sp.blk0[g + 1], Rp, s - g * R, o);
      if ((threadIdx.x & 31) == 0) fn(s, o);
    }
  } else {
    for (int s = (int)threadIdx.x; s < GR; s += nt) {
      if (skip(s)) continue;
      const int g = s / R, r = s - g * R;
      double2 o[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) o[c] = make_double2(0, 0);
      for (int b = sp.blk0[g]; b < sp.blk0[g + 1]; ++b)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const double2 v = __ldcg(reinterpret_cast<const double2*>(part) + ((size_t)b * Rp + r) * NC + c);
          o[c].x += v.x;
          o[c].y += v.y;
        }
      fn(s, o);
    }
  }
}

// For every global system s = g R + r: sum part[b][r] over the blocks b of
// segment g (reduce_systems); callback fn(s, sum).
template <class F>
__device__ __forceinline__ void reduce_partials(const double* part, const SegPlan& sp, int Rp, int R, F&& fn) {
  reduce_systems<1>(part, sp, R, Rp, [](int) { return false; }, [&](int s, const double2 (&o)[1]) { fn(s, o[0]); });
}


// one more SpMM for system s of segment s / R, if it is active (last block)
__device__ __forceinline__ void count_segment_iter(const KrylovState& ks, int s, int R) {
  if (ks.sys_iter && ks.active[s]) atomicAdd(ks.sys_iter + 1 + s / R, 1ULL);
}

// alpha = rho / <p, q> for system s (last block of a Krylov SpMM); a zero or
// non-finite <p, q> is a breakdown and freezes the system.
__device__ __forceinline__ void krylov_alpha(const KrylovState& ks, int s, double2 pq) {
  if (!ks.active[s]) {
    ks.alpha[2 * s] = 0;
    ks.alpha[2 * s + 1] = 0;
    return;
  }
  const double2 rho = make_double2(ks.rho[2 * s], ks.rho[2 * s + 1]);
  const double den = pq.x * pq.x + pq.y * pq.y;
  if (!(den > 0) || !isfinite(den)) {
    ks.alpha[2 * s] = 0;
    ks.alpha[2 * s + 1] = 0;
    ks.active[s] = 0;
    ks.status[s] = isfinite(den) ? BT_ENOCONV : BT_ENAN;
    atomicSub(ks.n_active, 1);
    return;
  }
  ks.alpha[2 * s] = (rho.x * pq.x + rho.y * pq.y) / den;
  ks.alpha[2 * s + 1] = (rho.y * pq.x - rho.x * pq.y) / den;
}

// End of one Krylov update for system s (last block): o[0] = rho' (complex),
// o[1].x = |r|^2.  Applies the convergence, stagnation and iteration-cap tests
// and forms beta = rho' / rho; returns whether the system stays active.
__device__ __forceinline__ bool krylov_step_finish(const KrylovState& ks, int s, const double2 (&o)[2],
                                                   int* pmode) {
  ks.rr[s] = o[1].x;
  const int it = ++ks.iter[s];
  if (!isfinite(o[1].x) || !isfinite(o[0].x) || !isfinite(o[0].y)) {
    ks.active[s] = 0;
    ks.status[s] = BT_ENAN;
    return false;
  }
  if (o[1].x <= ks.tol2[s]) {
    ks.active[s] = 0;
    return false;
  }
  if (o[1].x < ks.rr_best[s]) {
    ks.rr_best[s] = o[1].x;
    ks.it_best[s] = it;
  } else if (ks.stall > 0 && it - ks.it_best[s] >= ks.stall) {
    // the FP32 recurrence has stagnated: hand back to the refinement loop
    ks.active[s] = 0;
    if (pmode) pmode[s] = 0;
    return false;
  }
  if (it >= ks.max_iter) {
    ks.active[s] = 0;
    ks.status[s] = BT_ENOCONV;
    return false;
  }
  if (pmode && pmode[s]) {
    // polynomial-preconditioned system: rho and beta come from z = P_c r
    // (k_precond_dot); fall back to Jacobi when it is not converged within
    // 32 iterations (each costs nine SpMM-class launches; a useful
    // polynomial needs a few) or max_iter / 2 if that is fewer
    if (it >= min(ks.max_iter / 2, 32)) {
      ks.active[s] = 0;
      pmode[s] = 0;
      return false;
    }
    return true;
  }
  // beta = rho' / rho (complex)
  const double2 rho = make_double2(ks.rho[2 * s], ks.rho[2 * s + 1]);
  const double den = rho.x * rho.x + rho.y * rho.y;
  if (!(den > 0)) {
    ks.active[s] = 0;
    ks.status[s] = BT_ENOCONV;
    return false;
  }
  ks.beta[2 * s] = (o[0].x * rho.x + o[0].y * rho.y) / den;
  ks.beta[2 * s + 1] = (o[0].y * rho.x - o[0].x * rho.y) / den;
  ks.rho[2 * s] = o[0].x;
  ks.rho[2 * s + 1] = o[0].y;
  return true;
}

// Refinement bookkeeping of system s after a residual launch (last block).
// mode 0: step start, t = (|r_0|^2, |u|^2); mode 1: after a correction, t.x = |r|^2.
__device__ __forceinline__ void refine_finish(int mode, const RefineState& rf, int s, double2 t) {
  if (!rf.active[s]) return;
  if (mode == 0) {
    rf.r0n2[s] = t.x;
    rf.rk2[s] = t.x;
    rf.scale[s] = (double)(float)sqrt(t.x);  // FP32-exact: the same number scales and unscales
    if (!isfinite(t.x) || !isfinite(t.y)) {
      // a non-finite step residual: this system stops, the others go on
      rf.status[s] = BT_ENAN;
      rf.active[s] = 0;
      atomicSub(rf.n_active, 1);
    } else if (!(t.x > rf.floor_c2 * t.y)) {
      // nothing to solve: the increment is zero to FP64 rounding
      rf.active[s] = 0;
      atomicSub(rf.n_active, 1);
    }
  } else {
    const double prev = rf.rk2[s];
    if (!isfinite(t.x)) {
      rf.status[s] = BT_ENAN;
      rf.active[s] = 0;
      atomicSub(rf.n_active, 1);
      return;
    }
    rf.rk2[s] = t.x;
    rf.scale[s] = (double)(float)sqrt(t.x);
    // Converged; or stagnated near the rounding floor of the residual
    // arithmetic (a pass that no longer halves a residual already below
    // 1e-6 of the step's initial one): the achieved relative residual is what
    // err_est reports.  A pass that fails further up (the FP32 inner solve
    // stalled, e.g. at a near-breakdown of COCG, whose unconjugated (r, z) can
    // cancel when u's phase winds across the domain) is not a floor: the next
    // pass restarts the Krylov solve from the new residual, and a system still
    // unconverged when the passes run out is reported as BT_ENOCONV.
    const bool conv = !(t.x > rf.tol2 * rf.r0n2[s]);
    const bool floor = t.x > 0.25 * prev && t.x <= 1e-12 * rf.r0n2[s];
    if (conv || floor) {
      rf.err[s] += sqrt(t.x / rf.r0n2[s]);
      rf.active[s] = 0;
      atomicSub(rf.n_active, 1);
    }
  }
}
#endif

}  // namespace bt
