/*
 * bt.h -- C ABI of libbtgpu: GB300 (sm_103a) finite-element solver for the
 * multi-compartment Bloch-Torrey equation of diffusion MRI
 * (Nguyen, Li, Grebenkov, Hoffman et al., "Portable simulation framework for
 * diffusion MRI", arXiv 1908.01719).
 *
 * Method (paper section / equation):
 *   PDE      dU/dt = -i gamma f(t) g.x U + div(D grad U)        (Section 2, Eq. strong_BT)
 *   membrane flux continuity, mean flux = -kappa [U]            (Section 2, Eq. btpde_ic)
 *   outer    homogeneous Neumann, or pseudo-periodic             (Section 2, Eq. btpde_bc)
 *   profile  PGSE f(t), or any profile as F on the time grid     (Section 2, Eq. pgse;
 *                                                                 Section 3)
 *   signal   S = integral of U(x, TE) dx                         (Section 2, Eq. signal)
 *   b-value  b = gamma^2 |g|^2 int_0^TE F(s)^2 ds                (Section 2, Eq. b_value)
 *   space    P1 tetrahedra (or planar triangles, or the segments and surface
 *            triangles of thin tubes and layers), one nodal copy per compartment on
 *            interface nodes (PUFEM, Appendix A, Eq. phase_func)
 *   time     theta-method, matrix form A U^n = F                 (Appendix B, Eq. matrix_form)
 *   periodic gauge transform u = U exp(i gamma F(t) g.x)         (Appendix A, Eq. trBlo)
 *
 * Units: lengths in um, times in us (the paper's own convention).  With these
 * units D in mm^2/s, b in s/mm^2 and kappa in m/s keep their numerical values.
 *
 * Conventions for every entry point:
 *   - Return value: BT_OK (0) or a positive error code.  No C++ exception ever
 *     crosses the ABI.  After an error, bt_last_error(ctx) describes it.
 *   - Host pointers: read (or written) during the call only; the caller keeps
 *     ownership.  No entry point takes a device pointer unless it says so.
 *   - Device memory belongs to the context and is released by bt_destroy.
 *   - All device work is issued on the context's stream (default stream unless
 *     bt_set_stream was called); entry points that return results to host
 *     memory synchronise that stream before returning.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef BT_H
#define BT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int bt_status;
enum {
  BT_OK = 0,
  BT_EINVAL = 1,    /* invalid argument or mesh                              */
  BT_ENOMEM = 2,    /* host or device allocation failed                       */
  BT_ECUDA = 3,     /* CUDA runtime error (message in bt_last_error)          */
  BT_ENOCONV = 4,   /* a Krylov or refinement loop hit its iteration cap      */
  BT_ENAN = 5,      /* NaN/Inf met in a right-hand side or a Krylov scalar    */
  BT_ETIMEOUT = 6,  /* a slice SpMM block's wait for its tile copy ran past its
                       clock limit (about 2 s); the system's status records it */
  BT_ESTATE = 7,    /* call out of order (e.g. bt_run before bt_assemble)     */
  BT_ENODEV = 8     /* GPU call on a host-only context                        */
};

typedef struct bt_ctx bt_ctx;

/* Create a context on CUDA device `device`.  device < 0 creates a host-only
 * context: mesh upload, interface doubling, periodic identification and the
 * CSR pattern work (they run on the host), every GPU entry point returns
 * BT_ENODEV.  *out is set to NULL on failure. */
bt_status bt_create(bt_ctx** out, int device);
bt_status bt_destroy(bt_ctx* ctx);
/* Issue all device work on `cuda_stream` (a cudaStream_t; NULL = default). */
bt_status bt_set_stream(bt_ctx* ctx, void* cuda_stream);
const char* bt_last_error(const bt_ctx* ctx);

/* ---------------------------------------------------------------- mesh
 * Upload one geometry (copied).  xyz [3*n_nodes] (x,y,z per node, um);
 * tet4 [4*n_tets] node ids, positively oriented (signed volume > 0, else
 * BT_EINVAL); tet_cmpt [n_tets] compartment id in [0, n_cmpt);
 * D_cmpt [n_cmpt] diffusivity (um^2/us); kappa_cmpt [n_cmpt] membrane
 * permeability (um/us), +inf for "no membrane".  The face between
 * compartments a != b gets kappa = 1/(1/kappa_a + 1/kappa_b) (Eq. btpde_ic).
 * periodic_mask bit k: axis k periodic on [box_lo[k], box_hi[k]] (nodes on
 * the high face are identified with those on the low face, master-slave,
 * Eq. btpde_bc).  box_lo/box_hi also fix the origin of g.x: the box centre.
 * Builds, on the host: periodic identification, one dof per (node,
 * compartment) pair in increasing (master node, compartment) order,
 * interface faces and the shared CSR pattern of every matrix. */
bt_status bt_upload_mesh(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_tets,
                         const int32_t* tet4, const int32_t* tet_cmpt, int32_t n_cmpt,
                         const double* D_cmpt, const double* kappa_cmpt, uint32_t periodic_mask,
                         const double* box_lo, const double* box_hi);
/* The same for a 2-D domain (the paper's two-dimensional experiments, P1
 * triangles; Section 2 holds in any dimension): xy [2 n_nodes] (um), tri3
 * [3 n_tris] counter-clockwise triangles, tri_cmpt [n_tris]; periodic_mask
 * bits 0 (x) and 1 (y); box_lo, box_hi [2].  Internally the plane z = 0 of a
 * box [-1, 1] in z; gradient directions must lie in the xy plane
 * (bt_set_gradients refuses a z component with BT_EINVAL); interfaces are
 * edges with the jump term kappa <[u], [v]> on them.  Every later entry
 * point works unchanged; bt_set_weak_periodic couples boundary edges on the
 * x and y sides.  Errors as bt_upload_mesh (inverted triangles included). */
bt_status bt_upload_mesh_2d(bt_ctx* ctx, int64_t n_nodes, const double* xy, int64_t n_tris, const int32_t* tri3,
                            const int32_t* tri_cmpt, int32_t n_cmpt, const double* D_cmpt,
                            const double* kappa_cmpt, uint32_t periodic_mask, const double* box_lo,
                            const double* box_hi);
/* A 1-D manifold embedded in 3-D (Section 5, "Realistic neurons": simulation
 * on manifolds, after the thin-media method the paper cites; Section 1 on
 * the 1-D Bloch-Torrey equation of dendrite trees): the centre lines of thin
 * tubes as P1 segments, cross-sections taken uniform, so the weak form is
 * Section 2's with integrals along the curve and gradients tangential.
 * xyz [3 n_nodes] (um); seg2 [2 n_segs] node ids (any order; zero-length
 * segments are BT_EINVAL); seg_cmpt [n_segs] in [0, n_cmpt); D_cmpt
 * [n_cmpt].  Branch points are nodes shared by several segments.  No
 * membranes and no periodicity: segments of different compartments may not
 * share a node (BT_EINVAL).  box_lo/box_hi [3] fix the origin of g.x only.
 * Later calls work as for tetrahedra, in the lab frame only (bt_assemble
 * refuses BT_FRAME_TRANSFORMED: there |grad (q.x)|^2 would be (q.t)^2 per
 * segment, not q^2); bt_set_weak_periodic is refused. */
bt_status bt_upload_mesh_1d(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_segs, const int32_t* seg2,
                            const int32_t* seg_cmpt, int32_t n_cmpt, const double* D_cmpt, const double* box_lo,
                            const double* box_hi);
/* A thin layer as a 2-D manifold embedded in 3-D (Section 1's "thin-layer
 * and thin-tube media using a discretization on manifolds"; Section 5): P1
 * triangles of a surface, thickness taken uniform, so the weak form is
 * Section 2's with integrals over the surface and tangential gradients.
 * xyz [3 n_nodes] (um); tri3 [3 n_tris] node ids in any orientation
 * (zero-area triangles are BT_EINVAL); tri_cmpt [n_tris]; D_cmpt, kappa_cmpt
 * [n_cmpt] as for bt_upload_mesh: compartments meet along curves on the
 * surface, membranes there carry the jump term kappa <[u], [v]> per unit
 * length.  No periodicity; box_lo/box_hi [3] fix the origin of g.x only.
 * Lab frame only (bt_assemble refuses BT_FRAME_TRANSFORMED: there the
 * tangential part of q varies over the surface); bt_set_weak_periodic is
 * refused. */
bt_status bt_upload_mesh_surface(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_tris,
                                 const int32_t* tri3, const int32_t* tri_cmpt, int32_t n_cmpt, const double* D_cmpt,
                                 const double* kappa_cmpt, const double* box_lo, const double* box_hi);
/* Sizes after bt_upload_mesh.  Any output pointer may be NULL. */
bt_status bt_get_sizes(const bt_ctx* ctx, int64_t* n_dof, int64_t* nnz, int64_t* n_iface);
/* dof_node [n_dof] master node of each dof; dof_cmpt [n_dof] its compartment. */
bt_status bt_get_dofmap(const bt_ctx* ctx, int32_t* dof_node, int32_t* dof_cmpt);
/* CSR pattern: row_ptr [n_dof+1], col [nnz], columns ascending in each row. */
bt_status bt_get_pattern(const bt_ctx* ctx, int64_t* row_ptr, int32_t* col);
/* The halo tiles the shared-memory Krylov apply uses (host-side build, no GPU
 * needed): rows in Morton order of their node coordinates, cut into tiles of
 * at most 128 rows and 448 entries whose columns span at most `umax`
 * distinct rows.  With all
 * array pointers NULL only the sizes are returned (n_tiles, n_halo = total
 * halo entries).  Otherwise (caller-allocated): r0 [n_tiles+1] offsets into
 * rows; rows [n_dof] owned rows tile by tile; rowe [n_dof+1] first entry of
 * each owned row; rowl [n_dof] local halo index of each owned row; u0
 * [n_tiles+1] offsets into ucol; ucol [n_halo] halo rows ascending, bit 31 set
 * on the rows the tile owns; lidx [nnz] local column index of each entry in
 * tile order.  Tiles respect the current segments.  BT_EINVAL if umax is
 * outside [16, 65535] or a row has more than umax columns. */
bt_status bt_get_halo_tiles(bt_ctx* ctx, int32_t umax, int64_t* n_tiles, int64_t* n_halo, int32_t* r0,
                            int32_t* rows, int32_t* rowe, uint16_t* rowl, int32_t* u0, uint32_t* ucol,
                            uint16_t* lidx);

/* Transverse relaxation and initial magnetization per compartment (Section 2:
 * the T2 term of the Bloch-Torrey equation, which enters the weak form as
 * (U / T2, v), and the initial condition U(x, 0) = rho; Section 3 "Initial
 * conditions").  inv_T2 [n_cmpt] 1/T2 in 1/us (0 = no relaxation, the
 * default); rho [n_cmpt] initial value of u in that compartment (default 1).
 * Either pointer may be NULL (keeps the default).  The relaxation is
 * assembled into the operator as the plane MR = sum over elements of 1/T2 x
 * mass (bt_get_plane BT_PLANE_MR), so this call clears the assembly: call
 * bt_assemble (and the sequence and gradients) again.  BT_EINVAL for negative
 * or non-finite 1/T2 or non-finite rho. */
bt_status bt_set_relaxation(bt_ctx* ctx, const double* inv_T2, const double* rho);

/* Anisotropic diffusion (the diffusion term div(D grad U) of Section 2 with a
 * tensor D per compartment, as Section 3 "Diffusion coefficients and
 * tensors" allows): D6 [n_cmpt][6] = (xx, yy, zz, xy, yz, zx) in mm^2/s, each
 * symmetric positive semi-definite; NULL returns to the isotropic D_cmpt.
 * The tensor enters the stiffness K = (D grad phi_j, grad phi_i).  Lab frame
 * only (bt_assemble with BT_FRAME_TRANSFORMED then fails with BT_EINVAL: the
 * gauge-transformed operator would need direction-dependent D-weighted
 * masses).  Clears the assembly like bt_set_relaxation.  BT_EINVAL for
 * non-finite or indefinite tensors. */
bt_status bt_set_diffusion_tensor(bt_ctx* ctx, const double* D6);
/* Cell-based diffusion tensors (Section 3, "Diffusion coefficients and
 * tensors": d_jk cell-wise, set per cell from its midpoint or its marker):
 * D6 [n_elem][6] = (xx, yy, zz, xy, yz, zx) in mm^2/s for every element in
 * upload order, each finite and symmetric positive semi-definite; they
 * override the per-compartment tensors.  NULL removes them.  Lab frame only,
 * as bt_set_diffusion_tensor; clears the assembly.  BT_EINVAL names the first
 * non-finite or indefinite element. */
bt_status bt_set_element_tensors(bt_ctx* ctx, const double* D6);

/* Weak pseudo-periodic conditions on a box that is not meshed periodically
 * (Appendix B, "Weak implementation of the pseudo-periodic BCs"): on every
 * axis k of `axes` (bit mask, disjoint from the mesh's periodic_mask) the
 * faces x_k = lo_k and x_k = hi_k are coupled through an artificial
 * permeability kappa_e (um/us; <= 0 selects max D / h, h = (6 x mean
 * tetrahedron volume)^(1/3), or (2 x mean triangle area)^(1/2) in 2-D, where
 * the faces are boundary edges and axis z cannot be coupled).  Each step treats a face implicitly and its
 * partner face from the previous step with the phase e^{+-i q qhat_k L_k
 * F(t_n)}: L_n = M + theta dt (A_n + kappa_e B), r_0 += theta dt kappa_e C_n
 * u^{n-1}, B the boundary-face mass, C_n the face-mass coupling of partner
 * faces (Appendix B weighs the partner term by 1 - theta; theta is used for
 * both here, which is identical at theta = 1/2).  The two sides may be meshed
 * differently: a node's partner value is the opposite side's P1 field at the
 * node shifted by +-L_k e_k, interpolated in the face that contains that point
 * (the master/slave projection); on matching sides this is the node at the
 * shifted position.  BT_EINVAL if a shifted node falls outside the opposite
 * side.  Lab frame and one geometry only.  Clears the assembly like bt_set_relaxation; axes = 0
 * switches the coupling off.  BT_EINVAL for axes that are periodic in the
 * mesh, a 1-D manifold or a surface mesh. */
bt_status bt_set_weak_periodic(bt_ctx* ctx, uint32_t axes, double kappa_e);

/* ---------------------------------------------------------------- assembly
 * Element-by-element, deterministic assembly on the GPU of every matrix over
 * the shared pattern (Appendix B, Eq. matrix_form; Appendix A weak form):
 *   M mass, K stiffness (D-weighted), J interface (kappa-weighted),
 *   MD D-weighted mass, Mx My Mz first-moment mass (x relative to the box
 *   centre), Ex Ey Ez = C_k - C_k^T with C_k[i,j] = D int phi_i d_k phi_j,
 *   MR the 1/T2-weighted mass (zero without bt_set_relaxation),
 * then the step planes for time step dt_us and theta (0 < theta <= 1):
 *   A0 = M + theta dt (K + J + MR), in FP64, FP32 and double-float (hi+lo FP32).
 * flags: BT_FRAME_LAB (Neumann only) or BT_FRAME_TRANSFORMED (required when
 * periodic_mask != 0). */
enum { BT_FRAME_LAB = 0, BT_FRAME_TRANSFORMED = 1 };
bt_status bt_assemble(bt_ctx* ctx, double dt_us, double theta, uint32_t flags);
/* Copy one assembled FP64 value plane [nnz] to host memory. */
enum { BT_PLANE_M = 0, BT_PLANE_K = 1, BT_PLANE_J = 2, BT_PLANE_MD = 3, BT_PLANE_MX = 4,
       BT_PLANE_MY = 5, BT_PLANE_MZ = 6, BT_PLANE_EX = 7, BT_PLANE_EY = 8, BT_PLANE_EZ = 9,
       BT_PLANE_A0 = 10, BT_PLANE_MR = 11, BT_N_PLANES = 12 };
bt_status bt_get_plane(bt_ctx* ctx, int which, double* vals);

/* ---------------------------------------------------------------- sequence
 * PGSE (Eq. pgse): f = 1 on [0, delta], -1 on (Delta, Delta + delta], 0
 * otherwise; TE >= Delta + delta, TE/dt must be an integer (to 1e-9).  Each
 * theta step uses the step average of f on both sides (design reading of the
 * paper's f(t^n), f(t^{n-1})); F(t_n) is exact.  Needs bt_assemble first. */
enum {
  BT_PGSE = 0,
  BT_DOUBLE_PGSE = 1,      /* bt_set_waveform / bt_waveform_tables only (also below) */
  BT_COS_OGSE = 2,
  BT_SIN_OGSE = 3,
  BT_TRAPEZOID = 4,
  BT_DOUBLE_TRAPEZOID = 5
};
bt_status bt_set_sequence(bt_ctx* ctx, int kind, double delta_us, double Delta_us, double TE_us);
/* The tables of one of the paper's six temporal profiles (Section 3, "General
 * diffusion-encoding sequence"; the profiles compared in Section 4), with no
 * context: F [n_steps + 1] = F(t_n) = int_0^{t_n} f at t_n = n dt in closed
 * form (F[0] = 0) and int_F2 = int_0^TE F^2 (us^3, for b = q^2 int_F2,
 * Section 2 Eq. b_value) by composite Gauss-Legendre quadrature between the
 * profile's breakpoints.  Profiles (times in us):
 *   BT_PGSE              f = +1 on [0, delta], -1 on [Delta, Delta + delta]
 *   BT_DOUBLE_PGSE       two PGSE blocks, the second starting at Delta + delta
 *   BT_COS_OGSE          f = cos(w s) on [0, delta], -cos(w (s - tau)) on
 *                        (tau, tau + delta], w = 2 pi n_periods / delta,
 *                        tau = (delta + Delta) / 2
 *   BT_SIN_OGSE          the same with sin
 *   BT_TRAPEZOID         PGSE lobes with linear ramps of length ramp_us at both
 *                        ends (ramp_us <= 0: delta / 10)
 *   BT_DOUBLE_TRAPEZOID  two trapezoid blocks, the second at Delta + delta
 * n_steps (out, may be NULL) = TE / dt; F (may be NULL; n_steps + 1 doubles,
 * caller-owned) and int_F2 (may be NULL) are written when given.  BT_EINVAL
 * for an unknown kind, delta <= 0, Delta < delta, dt <= 0, TE not an integer
 * multiple of dt (to 1e-9), TE before the end of the profile, n_periods < 1
 * (OGSE) or a ramp longer than delta / 2. */
bt_status bt_waveform_tables(int kind, double delta_us, double Delta_us, double TE_us, double dt_us,
                             int32_t n_periods, double ramp_us, int32_t* n_steps, double* F, double* int_F2);
/* bt_set_profile with the tables of bt_waveform_tables for the context's dt
 * (BT_PGSE is bt_set_sequence).  Needs bt_assemble first; the same errors as
 * bt_waveform_tables and bt_set_profile. */
bt_status bt_set_waveform(bt_ctx* ctx, int kind, double delta_us, double Delta_us, double TE_us,
                          int32_t n_periods, double ramp_us);
/* Several geometries of uneven size in one context (the uneven batch): after
 * uploading their disjoint union as one mesh (nodes of geometry g =
 * [node_off[g], node_off[g+1]), every tetrahedron inside one geometry, each
 * geometry centred on the box centre so that g.x uses its own origin) and
 * assembling, give each geometry its PGSE timing.  The time loop then runs all
 * geometries together, each right-hand side set repeated per geometry, and
 * freezes a geometry after its own TE.  System (signal) index s = g R + r.
 * Replaces bt_set_sequence; call bt_set_gradients afterwards.  Lab frame or
 * Neumann transformed frame only (no periodic box). */
bt_status bt_set_segments(bt_ctx* ctx, int32_t G, const int64_t* node_off, const double* delta_us,
                          const double* Delta_us, const double* TE_us);
/* An arbitrary temporal profile f(t) (Section 3, "General diffusion-encoding
 * sequence"; the magnetization equation and b of Section 2, Eq. strong_BT and
 * Eq. b_value), given by its integral on the time grid:
 *   F [n_steps + 1]  F(t_n) = int_0^{t_n} f(s) ds at t_n = n dt (us), F[0] = 0;
 *   int_F2           int_0^TE F(s)^2 ds (us^3), TE = n_steps dt, used for
 *                    b = q^2 int_F2 in bt_set_gradients.
 * Each step uses the step average f_bar_n = (F_n - F_{n-1}) / dt (lab frame)
 * or F_n (transformed frame, which needs F(TE) = 0), as for PGSE.  Replaces
 * bt_set_sequence (one geometry; bt_set_segments stays PGSE); call
 * bt_set_gradients afterwards.  BT_EINVAL for F[0] != 0, non-finite values,
 * int_F2 <= 0, or F(TE) != 0 in the transformed frame. */
bt_status bt_set_profile(bt_ctx* ctx, int32_t n_steps, const double* F, double int_F2);
/* Directions dirs [3*n_dir] (normalised here) and b-values bvals [n_b]
 * (s/mm^2).  Right-hand side r = d*n_b + j uses dirs[d], bvals[j];
 * q = gamma |g| = sqrt(b / int_0^TE F^2) (Eq. b_value): delta^2 (Delta - delta/3)
 * for PGSE, the caller's int_F2 after bt_set_profile. */
bt_status bt_set_gradients(bt_ctx* ctx, int32_t n_dir, const double* dirs, int32_t n_b,
                           const double* bvals);

/* ---------------------------------------------------------------- solve
 * Modes:
 *   BT_MODE_PLAIN_FP64  FP64 vectors and Krylov (COCG in the lab frame, CG in
 *                       the transformed frame), Jacobi; stop at
 *                       |r| <= tol_fp64 * |r_0| per step.
 *   BT_MODE_MIXED       FP32 complex SpMM and Krylov vectors inside
 *                       iterative refinement; refinement residuals in
 *                       double-float (or native FP64 with BT_OPT_RESID_FP64);
 *                       stop at |r| <= tol_ref * |r_0|.
 *   BT_MODE_LEARNED     as MIXED, with the learned polynomial preconditioner
 *                       (bt_load_precond / bt_train_precond) or a fixed one
 *                       (bt_set_precond_poly) in the inner Krylov; Jacobi
 *                       fallback.
 * Each step solves L_n d = r_0 = (R_n - L_n) u^{n-1}, u^n = u^{n-1} + d, with
 * L_n = M + theta dt A_n, R_n = M - (1-theta) dt A_{n-1} (Appendix B). */
enum { BT_MODE_PLAIN_FP64 = 0, BT_MODE_MIXED = 1, BT_MODE_LEARNED = 2 };
/* Option flags: BT_OPT_RESID_FP64 native-FP64 refinement residuals;
 * BT_OPT_PROFILE CUDA events around every fused SpMM and residual launch
 * (host-driven loop); BT_OPT_NO_GRAPH host-driven loop instead of the
 * captured run graph (one launch per simulation: WHILE nodes over the time
 * steps, the refinement passes and the inner iterations); BT_OPT_VARIANT_ROW / _HALO bypass the autotuner and
 * use that Krylov variant together with the row / halo double-float residuals
 * (bt_get_tuning; _HALO falls back to the tuned choice where the halo tiles
 * are not available); BT_OPT_VARIANT_SLICE bypasses the autotuner's Krylov
 * choice for the slice-tiled iteration, the fastest of its configurations
 * (bt_get_tuning variants 2..6); BT_OPT_SLICE_ONE_STAGE forces configuration
 * 1 (variant 3), and (c + 1) << BT_OPT_SLICE_CONFIG_SHIFT forces
 * configuration c in 0..4 (variant 2 + c).  The residual kernel is still
 * tuned, and the slice flags fall back to the tuned choice when the padded
 * RHS width is not a multiple of 32 or a row does not fit the
 * configuration's tiles. */
enum {
  BT_OPT_RESID_FP64 = 1u,
  BT_OPT_PROFILE = 2u,
  BT_OPT_NO_GRAPH = 4u,
  BT_OPT_VARIANT_ROW = 8u,
  BT_OPT_VARIANT_HALO = 16u,
  BT_OPT_VARIANT_SLICE = 32u,
  BT_OPT_SLICE_ONE_STAGE = 64u,
  BT_OPT_SLICE_CONFIG_SHIFT = 8  /* bits 8..10: slice configuration + 1 (0 = none) */
};
typedef struct bt_solver_opts {
  double tol_fp64;      /* plain FP64 stopping tolerance (default 1e-12)          */
  double tol_inner;     /* inner FP32 Krylov tolerance (default 1e-4)             */
  double tol_ref;       /* refinement tolerance (default 1e-8)                    */
  int32_t max_iter;     /* Krylov iteration cap per solve (default 1000)          */
  int32_t max_refine;   /* refinement passes per step (default 6)                 */
  int32_t check_every;  /* host polls convergence every k iterations (default 4)  */
  uint32_t flags;       /* BT_OPT_*                                               */
  int32_t rhs_begin;    /* solve RHS [rhs_begin, rhs_end); both 0 = all           */
  int32_t rhs_end;
} bt_solver_opts;
/* Fill `o` with the defaults above. */
bt_status bt_default_opts(bt_solver_opts* o);
/* Run the whole time loop from u^0 = 1 to TE for the selected RHS. */
bt_status bt_run(bt_ctx* ctx, int mode, const bt_solver_opts* opts);
/* Results of the last bt_run, per system s = g R + r (G = 1 without
 * segments).  S_re_im [2 G R] (re, im, um^3); err_est [G R] sum over steps
 * of the final relative refinement residual |r|/|r_0| (an upper proxy of the
 * relative signal error); status [G R] BT_OK / BT_ENOCONV / BT_ENAN.  Any
 * pointer may be NULL. */
bt_status bt_get_signals(bt_ctx* ctx, double* S_re_im, double* err_est, int32_t* status);
/* The field u^N at TE of one system of the last bt_run (the discrete
 * magnetization of Appendix B's time loop, lab or transformed frame as
 * assembled), as FP64 complex values in the context's dof numbering
 * (bt_get_dofmap).  system = g R + r; with G = 1 it must lie in the RHS range
 * of the last run.  u_re_im [2 n_g] (re, im per dof) receives the dofs of
 * geometry g, n_g = node_off-derived dof count of that segment (n_dof when
 * G = 1); n_rows (may be NULL) receives n_g.  Mixed runs return hi + lo of the
 * double-float state rounded to FP64.  BT_ESTATE if no run left a state (any
 * call that changes the mesh, assembly, sequence, segments or gradients
 * discards it), BT_EINVAL for a system outside the last run. */
bt_status bt_get_state(bt_ctx* ctx, int32_t system, double* u_re_im, int64_t* n_rows);
/* The Krylov variant and residual kernel of the last FP32 run (the
 * autotuner's choice unless an option flag forced another) and the
 * autotuner's timings, made at the first FP32 run of a given RHS count,
 * RHS-per-lane and segmentation by timing one inner iteration of each
 * variant on the real pattern:
 *   0  row SpMM (one warp per row, X gathered per nonzero) + vector updates
 *   1  halo-staged apply (Morton-ordered row tiles, their halo rows of X staged
 *      in shared memory, search-direction and solution updates fused in) +
 *      z update; offered in BT_MODE_MIXED only
 *   2  slice-tiled apply (Morton tiles, one 32-system slice of the halo rows
 *      of p staged in shared memory, the tile's planes by TMA bulk copy)
 *      + r update (rho', |r|^2) + x and p update; offered in BT_MODE_MIXED
 *      when the padded RHS width is a multiple of 32.  Configuration 0:
 *      tiles of at most 256 halo rows, 128 owned rows and 1,536 entries, two
 *      pipelined stages, one block of 512 threads per SM
 *   3  configuration 1: the same tiles, one stage, two blocks of 256 per SM
 *   4  configuration 2: tiles of at most 128 halo rows, 64 owned rows and
 *      1,024 entries, two stages, two blocks of 256 per SM
 *   5  configuration 3: the small tiles, one stage, three blocks of 256 per SM
 *   6  configuration 4: the large tiles, two stages filled by one copy warp
 *      (cp.async halo rows, TMA planes, per-stage full/empty mbarriers), 15
 *      summing warps that take rows of a filled stage as they come; one
 *      block of 512 per SM
 * ms_iter [7] (may be NULL) receives the measured ms per iteration of each
 * (0 = not timed or not offered).  The double-float correction residual is tuned on its own:
 * resid_variant 0 = row kernel, 1 = halo-staged kernel (the step-start
 * residual follows it), ms_resid [2] the measured ms per launch of each.
 * Any pointer may be NULL.  BT_ESTATE before any tuning. */
bt_status bt_get_tuning(const bt_ctx* ctx, int32_t* variant, double* ms_iter, int32_t* resid_variant,
                        double* ms_resid);
/* Counters of the last bt_run (any pointer may be NULL): time steps, total
 * Krylov iterations (summed over solves, not RHS), refinement passes, fused
 * SpMM launches, with BT_OPT_PROFILE the summed device time (ms) of the
 * FP32/FP64 fused SpMM launches (for Krylov variant 1 the halo-staged apply)
 * and of the refinement-residual launches, the number of refinement-residual
 * launches and of all kernel launches, the number of active systems summed
 * over the fused SpMM launches (the right-hand sides each launch actually
 * processed), and with BT_OPT_PROFILE the summed device time (ms) of the
 * other kernels of the Krylov iterations (vector updates, inner products). */
/* The active systems of the last bt_run summed over its fused SpMM launches,
 * per segment (geometry): sys_iters [G], G = the context's segment count (1
 * without bt_set_segments).  With each segment's row count n_g this gives the
 * exact vector traffic of an uneven batch.  BT_EINVAL for another G or before
 * any run. */
bt_status bt_get_segment_stats(const bt_ctx* ctx, int32_t G, int64_t* sys_iters);
bt_status bt_get_stats(const bt_ctx* ctx, int64_t* steps, int64_t* krylov_iters,
                       int64_t* refine_passes, int64_t* spmm_launches, double* spmm_ms,
                       double* resid_ms, int64_t* resid_launches, int64_t* kernel_launches,
                       int64_t* sys_iters, double* vec_ms);

/* ---------------------------------------------------------------- learned preconditioner
 * A small network (5 -> 64 -> 64 -> 9, ReLU, bfloat16 weights, FP32
 * accumulation) maps the features of one step solve
 *   (dt [us], q|f_bar| [rad/(um us)] in the lab frame or q|F| [rad/um] in the
 *    transformed frame, D [um^2/us], kappa [um/us], h [um])
 * (each normalised as (log(x + eps) - mu)/sd with fixed constants) to the
 * coefficients c_0..c_8 of the polynomial preconditioner
 *   P_c = sum_j c_j (D^-1 L)^j D^-1,  D = diag(L), L the step matrix,
 * applied by Horner (8 fused SpMMs) inside the inner Krylov solve.  A system
 * falls back to Jacobi when the polynomial breaks down (rho = 0, or a
 * non-positive <r, z> for the Hermitian transformed systems), stagnates, or
 * has not converged within 32 iterations (max_iter / 2 if fewer); the
 * refinement tolerance judges the
 * result, so signals match the Jacobi path to that tolerance.  (The paper's
 * solver is unnamed, Appendix B; this preconditioner has no counterpart
 * there.)  Parameters: BT_PRECOND_NPARAM floats in the order W1 (64x5,
 * row-major), b1, W2 (64x64), b2, W3 (9x64), b3. */
enum { BT_PRECOND_NPARAM = 5 * 64 + 64 + 64 * 64 + 64 + 9 * 64 + 9 };
enum { BT_TRAIN_CONTINUE = 1u };
typedef struct bt_train_opts {
  int32_t epochs;   /* default 300  */
  int32_t batch;    /* default 512  */
  double lr;        /* Adam step (default 2e-3; betas 0.9, 0.999)       */
  uint64_t seed;    /* initialisation and shuffling (default 1)         */
  uint32_t flags;   /* BT_TRAIN_CONTINUE: start from the current weights */
  double rel_err;   /* relative accuracy of G and h (default 1e-6, the FP32
                       Krylov vectors of bt_collect_precond_data): the
                       objective adds the loss's spread
                       rel_err (2 |c|.|h| + |c|.|G| |c|) per sample; 0 = the
                       plain loss.  The Krylov basis is nearly dependent, so
                       without it the network can fit the data's rounding
                       (a small training loss that no solve sees). */
} bt_train_opts;
bt_status bt_train_default_opts(bt_train_opts* o);
/* Geometry features of the assembled mesh: volume-weighted mean D,
 * area-weighted mean interface kappa (0 without interfaces), and
 * h = (6 * mean tetrahedron volume)^(1/3). */
bt_status bt_precond_features(const bt_ctx* ctx, double* D, double* kappa, double* h);
/* Training samples from the method's own step solves: runs the mixed-mode time
 * loop (opts as bt_run) up to the last listed step (the context's signals are
 * then those of that step's state) and, at each listed step (1-based), takes every RHS's
 * normalised step residual r and the Krylov basis y_j = L (D^-1 L)^j D^-1 r,
 * j = 0..8, returning per sample (sample = step-major, then RHS):
 * feat [5], G = Re(Y^H Y)/|r|^2 [81], h = Re(Y^H r)/|r|^2 [9].
 * Output arrays hold n_steps * R samples. */
bt_status bt_collect_precond_data(bt_ctx* ctx, const bt_solver_opts* opts, int32_t n_steps, const int32_t* steps,
                                  float* feat, double* G, double* h);
/* Train on n samples (feat [n][5], G [n][81], h [n][9]) with minibatch Adam on
 * the mean loss |r - L P_c r|^2/|r|^2 = 1 - 2 c.h + c.G c plus rel_err times
 * its spread (bt_train_opts); loss_hist[epoch] (may be NULL) receives the
 * mean training objective of each epoch.  The network
 * stays in the context for BT_MODE_LEARNED. */
bt_status bt_train_precond(bt_ctx* ctx, int64_t n, const float* feat, const double* G, const double* h,
                           const bt_train_opts* opts, double* loss_hist);
/* Coefficients [n][9], mean objective and its gradient [BT_PRECOND_NPARAM]
 * of the current network on n samples (any output may be NULL; G, h needed
 * for loss and gradient): the mean loss plus rel_err times its spread, as in
 * training (rel_err = 0: the plain loss; BT_EINVAL outside [0, 1)). */
bt_status bt_precond_eval(bt_ctx* ctx, int64_t n, const float* feat, const double* G, const double* h,
                          double rel_err, double* coef, double* loss, double* grad);
/* Copy the FP32 master weights out / in (BT_PRECOND_NPARAM floats). */
bt_status bt_save_precond(const bt_ctx* ctx, float* w);
bt_status bt_load_precond(bt_ctx* ctx, const float* w);

/* ---------------------------------------------------------------- fixed polynomial baseline
 * The comparison the learned polynomial has to win: one fixed polynomial
 * P = sum_j c_j (D^-1 L)^j D^-1 for every system and step, applied by the
 * same Horner kernels.  (No counterpart in the paper, whose solver is
 * unnamed, Appendix B.)
 *
 * bt_set_precond_poly: c9 [9] host array, copied; BT_MODE_LEARNED then uses
 * these coefficients instead of the network (no network needed).  c9 = NULL
 * returns BT_MODE_LEARNED to the network.  BT_EINVAL for a non-finite
 * coefficient.
 *
 * bt_chebyshev_poly: the degree-8 p whose residual polynomial 1 - l p(l) is
 * T_9((hi + lo - 2 l)/(hi - lo)) / T_9((hi + lo)/(hi - lo)), T_9 the Chebyshev
 * polynomial of the first kind: the least maximum residual over [lo, hi]
 * among residual polynomials of degree 9 with value 1 at 0.  c9 [9] (out),
 * monomial coefficients in l.  BT_EINVAL unless 0 < lo < hi < inf.  Host
 * code; needs no context.
 *
 * bt_fit_chebyshev: the interval whose Chebyshev polynomial minimises the
 * mean of the per-sample loss 1 - 2 c.h + c.G c over n samples of
 * bt_collect_precond_data (G [n][81], h [n][9], host arrays), plus the
 * loss's uncertainty rel_err (2 |c|.|h| + |c|.|G| |c|) (means of the entry
 * moduli) for data known to relative accuracy rel_err (about 1e-6 for the
 * collected samples, whose Krylov vectors are FP32; the Krylov basis is close
 * to linearly dependent, so without it large coefficients can show a small
 * or negative loss).  hi is kept at or above 1.05 lam, lam = the largest
 * |y_8| / |y_7| over the samples (a power-iteration estimate of the largest
 * eigenvalue modulus of D^-1 L).  Search: a log-spaced grid over hi in
 * [max(1/4, 1.05 lam), max(16, 4.2 lam)] and lo/hi in [1e-4, 0.95], refined
 * three times around the best point.  Outputs (each may be NULL): lo, hi,
 * c9 [9], loss = the mean loss at the optimum (without the uncertainty term).
 * BT_EINVAL for n < 1, rel_err outside [0, 1) or non-finite data.
 *
 * bt_get_precond_stats: Horner launches of the last bt_run (each is one
 * fused SpMM over the polynomial systems). */
bt_status bt_set_precond_poly(bt_ctx* ctx, const double* c9);
bt_status bt_chebyshev_poly(double lo, double hi, double* c9);
bt_status bt_fit_chebyshev(int64_t n, const double* G, const double* h, double rel_err, double* lo, double* hi,
                           double* c9, double* loss);
bt_status bt_get_precond_stats(const bt_ctx* ctx, int64_t* horner_launches);

/* ---------------------------------------------------------------- allocation-free gradient
 * bt_precond_grad_noalloc computes what bt_precond_eval computes, with
 * rel_err = 0, for the loss and gradient of the preconditioner network, for
 * callers that cannot
 * allocate device memory: code under a framework that owns every device
 * allocation (a caching allocator or a fixed budget that cudaMalloc would
 * bypass), or a service that forbids allocation after start-up because
 * cudaMalloc and cudaFree synchronise the device.  It calls no cudaMalloc, cudaFree or allocating
 * library routine; its scratch is a fixed file-scope device array of about
 * 2.2 MB that every GPU loading the library holds until the process exits.
 * The paper has no counterpart of this entry point.
 *
 * All pointers are DEVICE pointers owned by the caller: w [BT_PRECOND_NPARAM]
 * FP32 weights (converted to bfloat16 inside), feat [n][5] raw features,
 * G [n][81], h [n][9] (FP32), grad [BT_PRECOND_NPARAM] (FP64, out), loss [n]
 * per-sample losses (FP32, out; their mean is bt_precond_eval's loss).
 * stream: a cudaStream_t (NULL = default stream); the call is asynchronous.
 * 1 <= n <= BT_NOALLOC_MAX_SAMPLES, else BT_EINVAL (nothing is launched).
 * The first call on a device looks up the scratch array's device address;
 * make that first call before any stream capture.  All calls on a device share
 * the scratch array, so calls that overlap on the GPU (different streams, no
 * ordering between them) race; order them on one stream.  No context is used:
 * errors are reported by the return code only.  BT_ECUDA without a launch if
 * a launch error is already pending on the calling thread (it is left
 * pending), or if one of this call's launches fails.  The scratch address is
 * cached per device for the life of the process: after cudaDeviceReset on a
 * device, do not call this entry point on that device again. */
enum { BT_NOALLOC_MAX_SAMPLES = 2048 };
bt_status bt_precond_grad_noalloc(const float* w, int32_t n, const float* feat, const float* G, const float* h,
                                  double* grad, float* loss, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BT_H */
