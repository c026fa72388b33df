// Context of libbtgpu (internal; the ABI sees only an opaque pointer).
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "bt_kernels.cuh"

namespace bt {
constexpr int N_COUNTERS = 16;
struct EventPair {
  cudaEvent_t a, b;
  int kind;  // 0 fused Krylov SpMM, 1 refinement residual, 2 vector kernels of a Krylov iteration
};
}  // namespace bt

struct bt_ctx {
  int device = -1;
  bool host_only = true;
  cudaStream_t stream = nullptr;
  int sms = 152;
  std::string err;

  bt::HostMesh mesh;
  bool have_mesh = false;

  // device copies of the mesh and the contribution lists
  bt::DBuf<double> d_xyz, d_D, d_face_kappa, d_geo, d_fcoef;
  // relaxation and initial condition per compartment (bt_set_relaxation)
  std::vector<double> cm_invT2, cm_rho, cm_Dten;  // cm_Dten empty: isotropic
  std::vector<double> el_Dten;                     // [n_elem][6] cell-based tensors (empty: none)
  bool have_rho = false;
  bt::DBuf<double> d_invT2, d_rho_dof, d_Dten, d_Dten_el;
  // weak pseudo-periodic box (bt_set_weak_periodic)
  uint32_t weak_axes = 0;
  double weak_kappa_in = 0, weak_kappa = 0;
  bt::WeakPeriodic weak;
  bt::DBuf<double> d_MB, d_ww, d_Fstep;
  bt::DBuf<int32_t> d_wrows, d_wptr, d_wcol;
  bt::DBuf<int8_t> d_wcode;
  bt::DBuf<int32_t> d_tets, d_cmpt, d_face_ta, d_tc, d_fc, d_rp, d_col;
  bt::DBuf<int8_t> d_face_lv;
  bt::DBuf<int64_t> d_tc_ptr, d_fc_ptr;
  // assembled planes
  bt::DBuf<double> d_planes, d_A0, d_KJ, d_w, d_diag_md64;
  bt::DBuf<double4> d_pk64, d_diag64;
  bt::DBuf<float4> d_pk32, d_pkhi, d_pklo, d_diag32;
  bt::DBuf<float> d_md32, d_diag_md32;
  bt::DBuf<float2> d_kjmd_hi, d_kjmd_lo;
  bool assembled = false;
  double dt = 0, theta = 0.5, wmax = 0;
  int transformed = 0;

  // sequence (segment 0 when the context holds several geometries)
  bool have_seq = false;
  double delta = 0, Delta = 0, TE = 0;
  int n_steps = 0;
  std::vector<double> fbar, F;  // fbar[n-1], n = 1..N; F[n], n = 0..N
  // segments: G geometries of one block-diagonal system (G = 1: the whole mesh)
  int G = 1;
  std::vector<int64_t> seg_row0{0, 0};          // [G+1] dof offsets
  std::vector<double> seg_delta, seg_Delta, seg_TE;
  std::vector<double> seg_intF2;                 // int_0^TE F^2 per segment (b = q^2 int F^2)
  std::vector<int> seg_N;                        // steps per segment
  std::vector<std::vector<double>> seg_fbar, seg_F;
  bt::DBuf<int> d_blk_seg, d_blk0, d_seg_N, d_ctl;
  cudaStream_t cap_stream[4] = {nullptr, nullptr, nullptr, nullptr};  // captures of the run graph
  bt::DBuf<int64_t> d_row0;
  int nblk = 0;
  int64_t planes_version = 0;  // bumped by every assembly
  // halo tiles of the shared-memory Krylov apply (one segmentation, one umax)
  bt::DBuf<int32_t> h_r0, h_rows, h_rowe, h_u0, h_e0, h_seg0, h_slot;
  bt::DBuf<uint16_t> h_rowl, h_lidx;
  bt::DBuf<uint32_t> h_ucol;
  bt::DBuf<float4> h_pkt;
  bt::DBuf<float> h_mdt;
  bt::DBuf<float4> h_dft;  // double-float planes in tile-entry order (3 per entry)
  std::vector<int64_t> halo_for;
  int halo_umax = 0;
  bool halo_ok = false;             // every row fits a tile of umax halo rows
  int64_t halo_planes_version = -1;
  bool halo_attr = false;
  // slice tiles of the slice-tiled iteration (owned rows longest first), one
  // set per tile class (SLICE_CONF), and the plan of tile blocks per
  // configuration (per segment, in proportion to its tiles)
  struct SliceTiles {
    bt::DBuf<int32_t> r0, rows, rowe, u0, e0, seg0, slot;
    bt::DBuf<uint16_t> rowl, lidx;
    bt::DBuf<uint32_t> ucol;
    bt::DBuf<float4> pkt;
    bt::DBuf<float> mdt;
    std::vector<int64_t> made_for;  // segment row starts the tiles were built for
    std::vector<int32_t> seg_tile0;
    bool ok = false;                // every row fits a tile of this class
    int64_t planes_version = -1;
  } slice_t[2];
  bool slice_attr = false;
  struct SlicePlan {
    bt::DBuf<int32_t> blk_seg, blk0;
    int nblk = 0, S = 0;  // tile blocks of the uploaded plan, slices it was made for
  } slice_plan[bt::SLICE_NCONF];
  struct Tuned {
    int R, nb, G;
    int variant;   // 0 row SpMM, 1 halo, 2 + c the slice-tiled iteration in configuration c
    double ms[2 + bt::SLICE_NCONF];  // one Krylov iteration of each variant (ms; 0 = not timed)
    double ms_resid[2];  // one correction residual launch: row, halo (0 = not timed)
    bool resid_halo = false;
  };
  std::vector<Tuned> tuned;
  int last_variant = -1, last_resid_halo = 0;  // what the last FP32 run used (flags may override the tuning)

  // gradients
  int n_dir = 0, n_b = 0, R = 0;
  std::vector<double> qhat_rhs, q_rhs;  // [3 G R], [G R]

  // run buffers
  bt::DBuf<double> d_q, d_qhat;
  bt::DBuf<bt::OpCoef> d_coef;
  bt::DBuf<double2> u64, r64, x64, rk64, p64, q64;
  bt::DBuf<float4> udf, rdf;
  bt::DBuf<float2> x32, r32, p32, q32, p32b;  // p32b: second p buffer of the halo iteration
  bt::DBuf<double> ks_rho, ks_alpha, ks_beta, ks_rr0, ks_rr, ks_tol2;
  bt::DBuf<int> ks_iter, ks_active, ks_status, n_active, ks_it_best;
  bt::DBuf<double> ks_rr_best;
  bt::DBuf<int> ks_pend, ks_par;
  bt::DBuf<unsigned long long> d_sys_iter;
  bt::DBuf<double> rf_r0n2, rf_rk2, rf_scale, rf_err;
  bt::DBuf<int> rf_active;
  bt::DBuf<double> red_part, d_S;
  bt::DBuf<unsigned int> red_counter;
  // u^N left by the last run: kind 0 none, 1 FP64 (u64), 2 double-float (udf);
  // its padded width, RHS per lane and RHS range
  int last_kind = 0, last_Rp = 0, last_nb = 1, last_rb = 0, last_Rs = 0;
  bt::DBuf<double2> d_state;
  int* h_flags = nullptr;  // pinned: [0] Krylov n_active, [1] refinement n_active

  // results
  std::vector<double> S, err_est;
  std::vector<int> status;
  int64_t st_steps = 0, st_iters = 0, st_refine = 0, st_spmm = 0, st_resid = 0, st_launches = 0, st_sys_iters = 0;
  double st_spmm_ms = 0, st_resid_ms = 0, st_vec_ms = 0;
  std::vector<unsigned long long> st_seg_sys_iters;  // active systems summed over SpMM launches, per segment
  std::vector<bt::EventPair> ev_pool;
  size_t ev_used = 0;

  // learned polynomial preconditioner
  bool have_precond = false;
  bool have_fixed_poly = false;  // bt_set_precond_poly: one polynomial for every system and step
  double fixed_poly[9] = {0};
  int64_t st_horner = 0;  // Horner launches of the last run (the polynomial's SpMMs)
  bt::DBuf<float> pw32, pm, pv, d_feat;
  bt::DBuf<__nv_bfloat16> pw16;
  bt::DBuf<double> d_coef9;
  bt::DBuf<float2> zA, zB, Vbuf;
  bt::DBuf<int> pmode;
  bt::DBuf<double> gram_part, gram_out;
  double feat_D = 0, feat_kappa = 0, feat_h = 0;  // geometry features (bt_assemble)
};

namespace bt {
inline bt_status fail(bt_ctx* c, bt_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
// The last line of defence of every entry point: no C++ exception crosses the
// C ABI.  Setting the message may itself fail under memory exhaustion.
inline bt_status guard_fail(bt_ctx* c, bt_status code, const char* what) noexcept {
  if (c) {
    try {
      c->err = what;
    } catch (...) {
    }
  }
  return code;
}
template <class T>
cudaError_t ensure(DBuf<T>& b, size_t n) {
  if (b.n >= n && b.p) return cudaSuccess;
  return b.alloc(n);
}
}  // namespace bt

// Closes an entry point written as a function-try-block.
#define BT_ABI_CATCH(ctx_)                                                                       \
  catch (const std::bad_alloc&) {                                                                \
    return bt::guard_fail(ctx_, BT_ENOMEM, "host allocation failed");                           \
  }                                                                                              \
  catch (const std::exception& e_) {                                                             \
    return bt::guard_fail(ctx_, BT_EINVAL, e_.what());                                           \
  }                                                                                              \
  catch (...) {                                                                                  \
    return bt::guard_fail(ctx_, BT_EINVAL, "unexpected exception");                             \
  }

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return bt::fail(ctx, e_ == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA,               \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

#define CKL()                                                                                    \
  do {                                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess) return bt::fail(ctx, BT_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)
