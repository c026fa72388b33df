// C ABI of libbtgpu (declared in include/bt.h): context, mesh upload,
// assembly, sequence, gradients, the time loop with iterative refinement, and
// result read-back.  All arithmetic of the method runs in the CUDA kernels of
// this library; this file only moves data and sequences launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "bt_ctx.h"

using namespace bt;

namespace bt {
void compute_geom_features(bt_ctx* ctx);
}


namespace {

template <class T>
cudaError_t upload(DBuf<T>& b, const std::vector<T>& h, cudaStream_t st) {
  cudaError_t e = b.alloc(h.size());
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

bool need_gpu(bt_ctx* ctx) { return ctx && !ctx->host_only; }

EventPair* ev_next(bt_ctx* ctx, int kind) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    EventPair e;
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(e);
  }
  EventPair* e = &ctx->ev_pool[ctx->ev_used++];
  e->kind = kind;
  return e;
}

void ev_harvest(bt_ctx* ctx) {
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ctx->ev_pool[i].a, ctx->ev_pool[i].b) == cudaSuccess) {
      if (ctx->ev_pool[i].kind == 0) ctx->st_spmm_ms += ms;
      else if (ctx->ev_pool[i].kind == 2) ctx->st_vec_ms += ms;
      else ctx->st_resid_ms += ms;
    }
  }
  ctx->ev_used = 0;
}

}  // namespace

extern "C" {

bt_status bt_create(bt_ctx** out, int device) {
  if (!out) return BT_EINVAL;
  *out = nullptr;
  bt_ctx* c = new (std::nothrow) bt_ctx();
  if (!c) return BT_ENOMEM;
  c->device = device;
  c->host_only = device < 0;
  if (!c->host_only) {
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&c->h_flags, 4 * sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = c->red_counter.alloc(N_COUNTERS);
    if (e == cudaSuccess) e = cudaMemset(c->red_counter.p, 0, N_COUNTERS * sizeof(unsigned int));
    if (e != cudaSuccess) {
      delete c;
      return BT_ECUDA;
    }
  }
  *out = c;
  return BT_OK;
}

bt_status bt_destroy(bt_ctx* ctx) {
  if (!ctx) return BT_OK;
  if (!ctx->host_only) {
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->ev_pool) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    for (auto& s : ctx->cap_stream)
      if (s) cudaStreamDestroy(s);
  }
  delete ctx;
  return BT_OK;
}

bt_status bt_set_stream(bt_ctx* ctx, void* s) {
  if (!ctx) return BT_EINVAL;
  ctx->stream = (cudaStream_t)s;
  return BT_OK;
}

const char* bt_last_error(const bt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static bt_status upload_mesh_nv(bt_ctx* ctx, int nv, int64_t n_nodes, const double* xyz, int64_t n_tets,
                                const int32_t* tet4, const int32_t* tet_cmpt, int32_t n_cmpt, const double* D_cmpt,
                                const double* kappa_cmpt, uint32_t periodic_mask, const double* box_lo,
                                const double* box_hi, bool surface = false) {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!xyz || !tet4 || !tet_cmpt || !D_cmpt || !kappa_cmpt || !box_lo || !box_hi || n_nodes <= 0 || n_tets <= 0 ||
      n_cmpt <= 0 || periodic_mask > 7)
    return fail(ctx, BT_EINVAL, "bt_upload_mesh: invalid argument");
  // the 32-bit index limits, checked before any caller array is read
  if (n_nodes >= (int64_t(1) << 31) || n_tets >= (int64_t(1) << 27))
    return fail(ctx, BT_EINVAL, "bt_upload_mesh: mesh too large for 32-bit element indexing");
  HostMesh& m = ctx->mesh;
  m = HostMesh();
  ctx->have_mesh = ctx->assembled = ctx->have_seq = false;
  try {
    m.nv = nv;
    m.surface = surface;
    m.n_nodes = n_nodes;
    m.n_tets = n_tets;
    m.n_cmpt = n_cmpt;
    m.xyz.assign(xyz, xyz + 3 * n_nodes);
    m.tets.assign(tet4, tet4 + (size_t)nv * n_tets);
    m.tet_cmpt.assign(tet_cmpt, tet_cmpt + n_tets);
    m.D.assign(D_cmpt, D_cmpt + n_cmpt);
    m.kappa.assign(kappa_cmpt, kappa_cmpt + n_cmpt);
    m.pmask = periodic_mask;
    for (int k = 0; k < 3; ++k) {
      m.lo[k] = box_lo[k];
      m.hi[k] = box_hi[k];
    }
    std::string msg;
    int st = build_host_mesh(m, msg);
    if (st) return fail(ctx, st, "bt_upload_mesh: " + msg);
    for (double kf : m.face_kappa)
      if (!std::isfinite(kf))
        return fail(ctx, BT_EINVAL, "bt_upload_mesh: two compartments without membrane (kappa = inf) touch");
  } catch (const std::bad_alloc&) {
    return fail(ctx, BT_ENOMEM, "bt_upload_mesh: host allocation failed");
  }
  ctx->have_mesh = true;
  ctx->G = 1;
  ctx->seg_row0 = {0, ctx->mesh.n_dof};
  ctx->cm_invT2.assign(n_cmpt, 0.0);
  ctx->cm_rho.assign(n_cmpt, 1.0);
  ctx->cm_Dten.clear();
  ctx->el_Dten.clear();
  ctx->weak_axes = 0;
  ctx->have_rho = false;
  if (ctx->host_only) return BT_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  CK(upload(ctx->d_xyz, m.xyz, st));
  CK(upload(ctx->d_tets, m.tets, st));
  CK(upload(ctx->d_cmpt, m.tet_cmpt, st));
  CK(upload(ctx->d_D, m.D, st));
  CK(upload(ctx->d_face_ta, m.face_ta, st));
  CK(upload(ctx->d_face_lv, m.face_lv, st));
  CK(upload(ctx->d_face_kappa, m.face_kappa, st));
  CK(upload(ctx->d_tc_ptr, m.tc_ptr, st));
  CK(upload(ctx->d_tc, m.tc, st));
  CK(upload(ctx->d_fc_ptr, m.fc_ptr, st));
  CK(upload(ctx->d_fc, m.fc, st));
  std::vector<int32_t> rp32(m.row_ptr.begin(), m.row_ptr.end());
  CK(upload(ctx->d_rp, rp32, st));
  CK(upload(ctx->d_col, m.col, st));
  CK(cudaStreamSynchronize(st));
  return BT_OK;
}

bt_status bt_upload_mesh(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_tets, const int32_t* tet4,
                         const int32_t* tet_cmpt, int32_t n_cmpt, const double* D_cmpt, const double* kappa_cmpt,
                         uint32_t periodic_mask, const double* box_lo, const double* box_hi) try {
  return upload_mesh_nv(ctx, 4, n_nodes, xyz, n_tets, tet4, tet_cmpt, n_cmpt, D_cmpt, kappa_cmpt, periodic_mask,
                        box_lo, box_hi);
} BT_ABI_CATCH(ctx)

bt_status bt_upload_mesh_2d(bt_ctx* ctx, int64_t n_nodes, const double* xy, int64_t n_tris, const int32_t* tri3,
                            const int32_t* tri_cmpt, int32_t n_cmpt, const double* D_cmpt, const double* kappa_cmpt,
                            uint32_t periodic_mask, const double* box_lo, const double* box_hi) try {
  if (!ctx) return BT_EINVAL;
  if (!xy || !box_lo || !box_hi || n_nodes <= 0 || n_nodes >= (int64_t(1) << 31) || periodic_mask > 3)
    return fail(ctx, BT_EINVAL, "bt_upload_mesh_2d: invalid argument");
  // the plane z = 0 inside a box centred on it, so z moments vanish
  std::vector<double> xyz(3 * (size_t)n_nodes, 0.0);
  for (int64_t i = 0; i < n_nodes; ++i) {
    xyz[3 * i] = xy[2 * i];
    xyz[3 * i + 1] = xy[2 * i + 1];
  }
  const double lo[3] = {box_lo[0], box_lo[1], -1.0}, hi[3] = {box_hi[0], box_hi[1], 1.0};
  return upload_mesh_nv(ctx, 3, n_nodes, xyz.data(), n_tris, tri3, tri_cmpt, n_cmpt, D_cmpt, kappa_cmpt,
                        periodic_mask, lo, hi);
} BT_ABI_CATCH(ctx)

bt_status bt_upload_mesh_1d(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_segs, const int32_t* seg2,
                            const int32_t* seg_cmpt, int32_t n_cmpt, const double* D_cmpt, const double* box_lo,
                            const double* box_hi) try {
  if (!ctx) return BT_EINVAL;
  if (n_cmpt <= 0 || n_cmpt > (1 << 20)) return fail(ctx, BT_EINVAL, "bt_upload_mesh_1d: invalid argument");
  // no membranes on a manifold: the permeabilities are never used
  const std::vector<double> no_kappa((size_t)n_cmpt, 0.0);
  return upload_mesh_nv(ctx, 2, n_nodes, xyz, n_segs, seg2, seg_cmpt, n_cmpt, D_cmpt, no_kappa.data(), 0, box_lo,
                        box_hi);
} BT_ABI_CATCH(ctx)

bt_status bt_upload_mesh_surface(bt_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_tris,
                                 const int32_t* tri3, const int32_t* tri_cmpt, int32_t n_cmpt, const double* D_cmpt,
                                 const double* kappa_cmpt, const double* box_lo, const double* box_hi) try {
  if (!ctx) return BT_EINVAL;
  return upload_mesh_nv(ctx, 3, n_nodes, xyz, n_tris, tri3, tri_cmpt, n_cmpt, D_cmpt, kappa_cmpt, 0, box_lo, box_hi,
                        true);
} BT_ABI_CATCH(ctx)

bt_status bt_get_sizes(const bt_ctx* ctx, int64_t* n_dof, int64_t* nnz, int64_t* n_iface) {
  if (!ctx || !ctx->have_mesh) return BT_ESTATE;
  if (n_dof) *n_dof = ctx->mesh.n_dof;
  if (nnz) *nnz = ctx->mesh.nnz;
  if (n_iface) *n_iface = ctx->mesh.n_face;
  return BT_OK;
}

bt_status bt_get_dofmap(const bt_ctx* ctx, int32_t* dof_node, int32_t* dof_cmpt) {
  if (!ctx || !ctx->have_mesh) return BT_ESTATE;
  if (dof_node) std::memcpy(dof_node, ctx->mesh.dof_node.data(), ctx->mesh.n_dof * sizeof(int32_t));
  if (dof_cmpt) std::memcpy(dof_cmpt, ctx->mesh.dof_cmpt.data(), ctx->mesh.n_dof * sizeof(int32_t));
  return BT_OK;
}

bt_status bt_get_pattern(const bt_ctx* ctx, int64_t* row_ptr, int32_t* col) {
  if (!ctx || !ctx->have_mesh) return BT_ESTATE;
  if (row_ptr) std::memcpy(row_ptr, ctx->mesh.row_ptr.data(), (ctx->mesh.n_dof + 1) * sizeof(int64_t));
  if (col) std::memcpy(col, ctx->mesh.col.data(), ctx->mesh.nnz * sizeof(int32_t));
  return BT_OK;
}

bt_status bt_get_halo_tiles(bt_ctx* ctx, int32_t umax, int64_t* n_tiles, int64_t* n_halo, int32_t* r0,
                            int32_t* rows, int32_t* rowe, uint16_t* rowl, int32_t* u0, uint32_t* ucol,
                            uint16_t* lidx) try {
  if (!ctx) return BT_EINVAL;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_get_halo_tiles: no mesh");
  if (umax < 16 || umax > 65535) return fail(ctx, BT_EINVAL, "bt_get_halo_tiles: umax outside [16, 65535]");
  HaloTiles t;
  build_halo_tiles(ctx->mesh, ctx->seg_row0, umax, HALO_TMAX, HALO_EMAX, t);
  if (t.too_wide) return fail(ctx, BT_EINVAL, "bt_get_halo_tiles: a row has more than umax columns");
  if (n_tiles) *n_tiles = (int64_t)t.r0.size() - 1;
  if (n_halo) *n_halo = (int64_t)t.ucol.size();
  auto put = [](auto* dst, const auto& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  put(r0, t.r0);
  put(rows, t.rows);
  put(rowe, t.rowe);
  put(rowl, t.rowl);
  put(u0, t.u0);
  put(ucol, t.ucol);
  put(lidx, t.lidx);
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_relaxation(bt_ctx* ctx, const double* inv_T2, const double* rho) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_set_relaxation: no mesh");
  const int nc = ctx->mesh.n_cmpt;
  std::vector<double> it(nc, 0.0), rh(nc, 1.0);
  for (int c = 0; c < nc; ++c) {
    if (inv_T2) it[c] = inv_T2[c];
    if (rho) rh[c] = rho[c];
    if (!(it[c] >= 0) || !std::isfinite(it[c]) || !std::isfinite(rh[c]))
      return fail(ctx, BT_EINVAL, "bt_set_relaxation: need finite 1/T2 >= 0 and finite rho");
  }
  ctx->cm_invT2 = it;
  ctx->cm_rho = rh;
  ctx->have_rho = false;
  for (double v : rh) ctx->have_rho |= v != 1.0;
  // the relaxation enters the assembled operator: assemble again
  ctx->assembled = ctx->have_seq = false;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_weak_periodic(bt_ctx* ctx, uint32_t axes, double kappa_e) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_set_weak_periodic: no mesh");
  if (axes > 7 || (axes & ctx->mesh.pmask) || !std::isfinite(kappa_e))
    return fail(ctx, BT_EINVAL, "bt_set_weak_periodic: axes must be a mask of non-periodic axes");
  if (axes) {
    std::string msg;
    WeakPeriodic wp;
    if (int st = build_weak_periodic(ctx->mesh, axes, wp, msg)) return fail(ctx, st, "bt_set_weak_periodic: " + msg);
    double dmax = 0;
    for (double d : ctx->mesh.D) dmax = std::max(dmax, d);
    ctx->weak = std::move(wp);
    ctx->weak_kappa = kappa_e > 0 ? kappa_e : dmax / ctx->weak.h;  // max D / h by default
  }
  ctx->weak_axes = axes;
  ctx->weak_kappa_in = kappa_e;
  ctx->assembled = ctx->have_seq = false;
  return BT_OK;
} BT_ABI_CATCH(ctx)

// A symmetric tensor (xx, yy, zz, xy, yz, zx) that is finite and positive
// semi-definite: the leading minors of [[xx, xy, zx], [xy, yy, yz], [zx, yz, zz]]
// and the diagonal are non-negative (to rounding).
static bool tensor_ok(const double* d) {
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(d[k])) return false;
  const double m1 = d[0], m2 = d[0] * d[1] - d[3] * d[3];
  const double m3 = d[0] * (d[1] * d[2] - d[4] * d[4]) - d[3] * (d[3] * d[2] - d[4] * d[5]) +
                    d[5] * (d[3] * d[4] - d[1] * d[5]);
  const double sc = std::max({std::fabs(d[0]), std::fabs(d[1]), std::fabs(d[2]), 1e-300});
  return !(m1 < 0 || d[1] < 0 || d[2] < 0 || m2 < -1e-12 * sc * sc || m3 < -1e-12 * sc * sc * sc);
}

bt_status bt_set_diffusion_tensor(bt_ctx* ctx, const double* D6) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_set_diffusion_tensor: no mesh");
  const int nc = ctx->mesh.n_cmpt;
  if (!D6) {
    ctx->cm_Dten.clear();
  } else {
    std::vector<double> t(D6, D6 + 6 * (size_t)nc);
    for (int c = 0; c < nc; ++c)
      if (!tensor_ok(&t[6 * (size_t)c]))
        return fail(ctx, BT_EINVAL, "bt_set_diffusion_tensor: non-finite or indefinite tensor");
    ctx->cm_Dten = t;
  }
  ctx->assembled = ctx->have_seq = false;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_element_tensors(bt_ctx* ctx, const double* D6) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_set_element_tensors: no mesh");
  const int64_t ne = ctx->mesh.n_tets;
  if (!D6) {
    ctx->el_Dten.clear();
  } else {
    std::vector<double> t(D6, D6 + 6 * (size_t)ne);
    for (int64_t e = 0; e < ne; ++e)
      if (!tensor_ok(&t[6 * (size_t)e]))
        return fail(ctx, BT_EINVAL, "bt_set_element_tensors: non-finite or indefinite tensor at element " +
                                        std::to_string(e));
    ctx->el_Dten = std::move(t);
  }
  ctx->assembled = ctx->have_seq = false;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_assemble(bt_ctx* ctx, double dt_us, double theta, uint32_t flags) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_mesh) return fail(ctx, BT_ESTATE, "bt_assemble: no mesh");
  if (!need_gpu(ctx)) return fail(ctx, BT_ENODEV, "bt_assemble: host-only context");
  if (!(dt_us > 0) || !std::isfinite(dt_us) || !(theta > 0) || theta > 1 || flags > 1)
    return fail(ctx, BT_EINVAL, "bt_assemble: need dt > 0, 0 < theta <= 1, flags in {LAB, TRANSFORMED}");
  if (ctx->mesh.pmask && flags != BT_FRAME_TRANSFORMED)
    return fail(ctx, BT_EINVAL, "bt_assemble: periodic boxes need BT_FRAME_TRANSFORMED");
  if ((ctx->mesh.nv == 2 || ctx->mesh.surface) && flags != BT_FRAME_LAB)
    return fail(ctx, BT_EINVAL, "bt_assemble: manifold meshes need the lab frame");
  if ((!ctx->cm_Dten.empty() || !ctx->el_Dten.empty()) && flags == BT_FRAME_TRANSFORMED)
    return fail(ctx, BT_EINVAL, "bt_assemble: diffusion tensors need the lab frame");
  if (ctx->weak_axes && flags == BT_FRAME_TRANSFORMED)
    return fail(ctx, BT_EINVAL, "bt_assemble: the weak periodic box needs the lab frame");
  CK(cudaSetDevice(ctx->device));
  const HostMesh& m = ctx->mesh;
  const int64_t nnz = m.nnz, n = m.n_dof;
  cudaStream_t st = ctx->stream;
  CK(ctx->d_geo.alloc(33 * (size_t)m.n_tets));
  CK(ctx->d_fcoef.alloc(std::max<int64_t>(1, m.n_face)));
  CK(ctx->d_planes.alloc(11 * (size_t)nnz));
  CK(upload(ctx->d_invT2, ctx->cm_invT2, st));
  if (ctx->weak_axes) {
    std::vector<double> mb(ctx->weak.B);
    for (double& v : mb) v *= ctx->weak_kappa;
    CK(upload(ctx->d_MB, mb, st));
    CK(upload(ctx->d_wrows, ctx->weak.rows, st));
    CK(upload(ctx->d_wptr, ctx->weak.ptr, st));
    CK(upload(ctx->d_wcol, ctx->weak.col, st));
    CK(upload(ctx->d_ww, ctx->weak.w, st));
    CK(upload(ctx->d_wcode, ctx->weak.code, st));
  }
  if (!ctx->cm_Dten.empty()) CK(upload(ctx->d_Dten, ctx->cm_Dten, st));
  else ctx->d_Dten.free();
  if (!ctx->el_Dten.empty()) CK(upload(ctx->d_Dten_el, ctx->el_Dten, st));
  else ctx->d_Dten_el.free();
  if (ctx->have_rho) {
    std::vector<double> rd(n);
    for (int64_t i = 0; i < n; ++i) rd[i] = ctx->cm_rho[m.dof_cmpt[i]];
    CK(upload(ctx->d_rho_dof, rd, st));
  } else {
    ctx->d_rho_dof.free();
  }
  AsmArgs a{};
  a.xyz = ctx->d_xyz.p;
  a.tets = ctx->d_tets.p;
  a.cmpt = ctx->d_cmpt.p;
  a.Dc = ctx->d_D.p;
  a.invT2c = ctx->d_invT2.p;
  a.Dten = ctx->cm_Dten.empty() ? nullptr : ctx->d_Dten.p;
  a.DtenE = ctx->el_Dten.empty() ? nullptr : ctx->d_Dten_el.p;
  for (int k = 0; k < 3; ++k) a.centre[k] = 0.5 * (m.lo[k] + m.hi[k]);
  a.nt = m.n_tets;
  a.nv = m.nv;
  a.surface = m.surface ? 1 : 0;
  a.nf = m.n_face;
  a.nnz = nnz;
  a.face_ta = ctx->d_face_ta.p;
  a.face_lv = ctx->d_face_lv.p;
  a.face_kappa = ctx->d_face_kappa.p;
  a.tc_ptr = ctx->d_tc_ptr.p;
  a.tc = ctx->d_tc.p;
  a.fc_ptr = ctx->d_fc_ptr.p;
  a.fc = ctx->d_fc.p;
  a.geo = ctx->d_geo.p;
  a.fcoef = ctx->d_fcoef.p;
  a.planes = ctx->d_planes.p;
  launch_assembly(a, st);
  CKL();
  CK(ctx->d_A0.alloc(nnz));
  CK(ctx->d_KJ.alloc(nnz));
  CK(ctx->d_pk64.alloc(nnz));
  CK(ctx->d_pk32.alloc(nnz));
  CK(ctx->d_md32.alloc(nnz));
  CK(ctx->d_pkhi.alloc(nnz));
  CK(ctx->d_pklo.alloc(nnz));
  CK(ctx->d_kjmd_hi.alloc(nnz));
  CK(ctx->d_kjmd_lo.alloc(nnz));
  CK(ctx->d_w.alloc(n));
  CK(ctx->d_diag64.alloc(n));
  CK(ctx->d_diag_md64.alloc(n));
  CK(ctx->d_diag32.alloc(n));
  CK(ctx->d_diag_md32.alloc(n));
  DeriveArgs d;
  d.planes = ctx->d_planes.p;
  d.nnz = nnz;
  d.n = n;
  d.thdt = theta * dt_us;
  d.transformed = (int)flags;
  d.rp = ctx->d_rp.p;
  d.col = ctx->d_col.p;
  d.A0 = ctx->d_A0.p;
  d.KJ = ctx->d_KJ.p;
  d.pk64 = ctx->d_pk64.p;
  d.pk32 = ctx->d_pk32.p;
  d.md32 = ctx->d_md32.p;
  d.pkhi = ctx->d_pkhi.p;
  d.pklo = ctx->d_pklo.p;
  d.kjmd_hi = ctx->d_kjmd_hi.p;
  d.kjmd_lo = ctx->d_kjmd_lo.p;
  d.w = ctx->d_w.p;
  d.diag64 = ctx->d_diag64.p;
  d.diag_md64 = ctx->d_diag_md64.p;
  d.diag32 = ctx->d_diag32.p;
  d.diag_md32 = ctx->d_diag_md32.p;
  d.MB = ctx->weak_axes ? ctx->d_MB.p : nullptr;
  d.theta = theta;
  launch_derive(d, st);
  CKL();
  std::vector<double> w(n);
  CK(cudaMemcpyAsync(w.data(), ctx->d_w.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->wmax = 0;
  for (double x : w) ctx->wmax = std::max(ctx->wmax, std::fabs(x));
  ctx->dt = dt_us;
  ctx->theta = theta;
  ctx->transformed = (int)flags;
  compute_geom_features(ctx);
  ++ctx->planes_version;
  ctx->assembled = true;
  ctx->have_seq = false;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_get_plane(bt_ctx* ctx, int which, double* vals) try {
  if (!ctx || !vals || which < 0 || which >= BT_N_PLANES) return fail(ctx, BT_EINVAL, "bt_get_plane: bad argument");
  if (!need_gpu(ctx)) return fail(ctx, BT_ENODEV, "bt_get_plane: host-only context");
  if (!ctx->assembled) return fail(ctx, BT_ESTATE, "bt_get_plane: not assembled");
  CK(cudaSetDevice(ctx->device));
  const size_t plane = which == BT_PLANE_MR ? 10 : (size_t)which;
  const double* src = which == BT_PLANE_A0 ? ctx->d_A0.p : ctx->d_planes.p + plane * ctx->mesh.nnz;
  CK(cudaMemcpyAsync(vals, src, ctx->mesh.nnz * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_sequence(bt_ctx* ctx, int kind, double delta, double Delta, double TE) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->assembled) return fail(ctx, BT_ESTATE, "bt_set_sequence: assemble first (dt is needed)");
  if (kind != BT_PGSE) return fail(ctx, BT_EINVAL, "bt_set_sequence: only BT_PGSE");
  if (!(delta > 0) || !(Delta >= delta) || !(TE >= Delta + delta - 1e-9 * TE))
    return fail(ctx, BT_EINVAL, "bt_set_sequence: need 0 < delta <= Delta and TE >= Delta + delta");
  double ns = TE / ctx->dt;
  int N = (int)std::llround(ns);
  if (std::fabs(ns - N) > 1e-9 * std::max(1.0, ns) || N < 1)
    return fail(ctx, BT_EINVAL, "bt_set_sequence: TE must be an integer multiple of dt");
  ctx->delta = delta;
  ctx->Delta = Delta;
  ctx->TE = TE;
  ctx->n_steps = N;
  // F(t) = int_0^t f for PGSE; f_bar_n = (F(t_n) - F(t_{n-1})) / dt (step average)
  auto Ft = [&](double t) {
    double a = std::min(std::max(t, 0.0), delta);
    double b = std::min(std::max(t - Delta, 0.0), delta);
    return a - b;
  };
  ctx->F.resize(N + 1);
  ctx->fbar.resize(N);
  for (int n = 0; n <= N; ++n) ctx->F[n] = Ft(n * ctx->dt);
  for (int n = 1; n <= N; ++n) ctx->fbar[n - 1] = (ctx->F[n] - ctx->F[n - 1]) / ctx->dt;
  if (ctx->transformed && std::fabs(ctx->F[N]) > 1e-12 * delta)
    return fail(ctx, BT_EINVAL, "bt_set_sequence: F(TE) != 0 in the transformed frame");
  ctx->G = 1;
  ctx->seg_row0 = {0, ctx->mesh.n_dof};
  ctx->seg_delta = {delta};
  ctx->seg_Delta = {Delta};
  ctx->seg_intF2 = {delta * delta * (Delta - delta / 3.0)};  // int_0^TE F^2 for PGSE
  ctx->seg_TE = {TE};
  ctx->seg_N = {N};
  ctx->seg_fbar = {ctx->fbar};
  ctx->seg_F = {ctx->F};
  ctx->have_seq = true;
  ctx->R = 0;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_profile(bt_ctx* ctx, int32_t n_steps, const double* F, double int_F2) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->assembled) return fail(ctx, BT_ESTATE, "bt_set_profile: assemble first (dt is needed)");
  if (n_steps < 1 || !F) return fail(ctx, BT_EINVAL, "bt_set_profile: need n_steps >= 1 and F");
  if (!(int_F2 > 0) || !std::isfinite(int_F2)) return fail(ctx, BT_EINVAL, "bt_set_profile: need int_F2 > 0");
  double fmax = 0;
  for (int n = 0; n <= n_steps; ++n) {
    if (!std::isfinite(F[n])) return fail(ctx, BT_EINVAL, "bt_set_profile: non-finite F");
    fmax = std::max(fmax, std::fabs(F[n]));
  }
  if (F[0] != 0.0) return fail(ctx, BT_EINVAL, "bt_set_profile: F(0) must be 0");
  if (ctx->transformed && std::fabs(F[n_steps]) > 1e-12 * std::max(fmax, 1e-300))
    return fail(ctx, BT_EINVAL, "bt_set_profile: F(TE) != 0 in the transformed frame");
  const int N = n_steps;
  ctx->n_steps = N;
  ctx->TE = N * ctx->dt;
  ctx->delta = ctx->Delta = 0;
  ctx->F.assign(F, F + N + 1);
  ctx->fbar.resize(N);
  for (int n = 1; n <= N; ++n) ctx->fbar[n - 1] = (ctx->F[n] - ctx->F[n - 1]) / ctx->dt;
  ctx->G = 1;
  ctx->seg_row0 = {0, ctx->mesh.n_dof};
  ctx->seg_delta = {0.0};
  ctx->seg_Delta = {0.0};
  ctx->seg_TE = {ctx->TE};
  ctx->seg_intF2 = {int_F2};
  ctx->seg_N = {N};
  ctx->seg_fbar = {ctx->fbar};
  ctx->seg_F = {ctx->F};
  ctx->have_seq = true;
  ctx->R = 0;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_waveform(bt_ctx* ctx, int kind, double delta, double Delta, double TE, int32_t n_periods,
                          double ramp) try {
  if (!ctx) return BT_EINVAL;
  if (!ctx->assembled) return fail(ctx, BT_ESTATE, "bt_set_waveform: assemble first (dt is needed)");
  if (kind == BT_PGSE) return bt_set_sequence(ctx, kind, delta, Delta, TE);
  int32_t N = 0;
  if (bt_waveform_tables(kind, delta, Delta, TE, ctx->dt, n_periods, ramp, &N, nullptr, nullptr) != BT_OK)
    return fail(ctx, BT_EINVAL, "bt_set_waveform: invalid profile parameters (see bt_waveform_tables)");
  std::vector<double> F((size_t)N + 1);
  double I = 0;
  bt_waveform_tables(kind, delta, Delta, TE, ctx->dt, n_periods, ramp, &N, F.data(), &I);
  return bt_set_profile(ctx, N, F.data(), I);
} BT_ABI_CATCH(ctx)

bt_status bt_set_gradients(bt_ctx* ctx, int32_t n_dir, const double* dirs, int32_t n_b, const double* bvals) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->have_seq) return fail(ctx, BT_ESTATE, "bt_set_gradients: set the sequence first");
  if (n_dir <= 0 || n_b <= 0 || !dirs || !bvals || (int64_t)n_dir * n_b > 1024)
    return fail(ctx, BT_EINVAL, "bt_set_gradients: need 1 <= n_dir * n_b <= 1024");
  const int R = n_dir * n_b, G = ctx->G;
  std::vector<double> qh(3 * (size_t)G * R), qv((size_t)G * R);
  for (int g = 0; g < G; ++g) {
    const double intF2 = ctx->seg_intF2[g];
    for (int i = 0; i < n_dir; ++i) {
      double nx = dirs[3 * i], ny = dirs[3 * i + 1], nz = dirs[3 * i + 2];
      double nr = std::sqrt(nx * nx + ny * ny + nz * nz);
      if (!(nr > 0) || !std::isfinite(nr)) return fail(ctx, BT_EINVAL, "bt_set_gradients: zero direction");
      if (ctx->mesh.nv == 3 && !ctx->mesh.surface && std::fabs(nz) > 1e-12 * nr)
        return fail(ctx, BT_EINVAL, "bt_set_gradients: 2-D meshes need directions in the xy plane");
      for (int j = 0; j < n_b; ++j) {
        if (!(bvals[j] >= 0) || !std::isfinite(bvals[j])) return fail(ctx, BT_EINVAL, "bt_set_gradients: b < 0");
        const size_t s = (size_t)g * R + i * n_b + j;
        qh[3 * s] = nx / nr;
        qh[3 * s + 1] = ny / nr;
        qh[3 * s + 2] = nz / nr;
        qv[s] = std::sqrt(bvals[j] / intF2);  // b = q^2 int F^2 (Eq. b_value)
      }
    }
  }
  ctx->n_dir = n_dir;
  ctx->n_b = n_b;
  ctx->R = R;
  ctx->qhat_rhs = qh;
  ctx->q_rhs = qv;
  ctx->S.assign(2 * (size_t)G * R, 0.0);
  ctx->err_est.assign((size_t)G * R, 0.0);
  ctx->status.assign((size_t)G * R, BT_OK);
  return BT_OK;
} BT_ABI_CATCH(ctx)

// Several geometries in one context: segment g = nodes [node_off[g],
// node_off[g+1]) with its own PGSE timing; the time loop runs to the largest
// TE and freezes each segment after its own last step.
bt_status bt_set_segments(bt_ctx* ctx, int32_t G, const int64_t* node_off, const double* delta,
                          const double* Delta, const double* TE) try {
  if (!ctx) return BT_EINVAL;
  ctx->last_kind = 0;
  if (!ctx->assembled) return fail(ctx, BT_ESTATE, "bt_set_segments: assemble first");
  if (G < 1 || !node_off || !delta || !Delta || !TE) return fail(ctx, BT_EINVAL, "bt_set_segments: bad arguments");
  const HostMesh& m = ctx->mesh;
  if (m.pmask) return fail(ctx, BT_EINVAL, "bt_set_segments: periodic boxes hold one geometry");
  if (node_off[0] != 0 || node_off[G] != m.n_nodes) return fail(ctx, BT_EINVAL, "bt_set_segments: node offsets must cover the mesh");
  for (int g = 0; g < G; ++g)
    if (node_off[g + 1] <= node_off[g]) return fail(ctx, BT_EINVAL, "bt_set_segments: empty segment");
  // every tetrahedron inside one segment
  for (int64_t t = 0; t < m.n_tets; ++t) {
    const int32_t v0 = m.tets[m.nv * t];
    const int g = (int)(std::upper_bound(node_off, node_off + G + 1, (int64_t)v0) - node_off) - 1;
    for (int a2 = 1; a2 < m.nv; ++a2)
      if (m.tets[m.nv * t + a2] < node_off[g] || m.tets[m.nv * t + a2] >= node_off[g + 1])
        return fail(ctx, BT_EINVAL, "bt_set_segments: a tetrahedron spans two segments");
  }
  std::vector<int64_t> row0(G + 1);
  for (int g = 0; g <= G; ++g)
    row0[g] = std::lower_bound(m.dof_node.begin(), m.dof_node.end(), (int32_t)std::min<int64_t>(node_off[g], INT32_MAX)) -
              m.dof_node.begin();
  row0[G] = m.n_dof;
  for (int g = 0; g < G; ++g)
    if (row0[g + 1] <= row0[g]) return fail(ctx, BT_EINVAL, "bt_set_segments: segment without dofs");
  std::vector<int> N(G);
  std::vector<std::vector<double>> fb(G), FF(G);
  for (int g = 0; g < G; ++g) {
    const double d = delta[g], D = Delta[g], T = TE[g];
    if (!(d > 0) || !(D >= d) || !(T >= D + d - 1e-9 * T))
      return fail(ctx, BT_EINVAL, "bt_set_segments: need 0 < delta <= Delta and TE >= Delta + delta");
    const double ns = T / ctx->dt;
    N[g] = (int)std::llround(ns);
    if (std::fabs(ns - N[g]) > 1e-9 * std::max(1.0, ns) || N[g] < 1)
      return fail(ctx, BT_EINVAL, "bt_set_segments: TE must be an integer multiple of dt");
    auto Ft = [&](double t) {
      double a3 = std::min(std::max(t, 0.0), d);
      double b3 = std::min(std::max(t - D, 0.0), d);
      return a3 - b3;
    };
    FF[g].resize(N[g] + 1);
    fb[g].resize(N[g]);
    for (int n = 0; n <= N[g]; ++n) FF[g][n] = Ft(n * ctx->dt);
    for (int n = 1; n <= N[g]; ++n) fb[g][n - 1] = (FF[g][n] - FF[g][n - 1]) / ctx->dt;
  }
  ctx->G = G;
  ctx->seg_row0 = row0;
  ctx->seg_delta.assign(delta, delta + G);
  ctx->seg_Delta.assign(Delta, Delta + G);
  ctx->seg_intF2.resize(G);
  for (int g = 0; g < G; ++g) ctx->seg_intF2[g] = delta[g] * delta[g] * (Delta[g] - delta[g] / 3.0);
  ctx->seg_TE.assign(TE, TE + G);
  ctx->seg_N = N;
  ctx->seg_fbar = fb;
  ctx->seg_F = FF;
  ctx->delta = delta[0];
  ctx->Delta = Delta[0];
  ctx->TE = TE[0];
  ctx->n_steps = *std::max_element(N.begin(), N.end());
  ctx->fbar = fb[0];
  ctx->F = FF[0];
  ctx->have_seq = true;
  ctx->R = 0;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_default_opts(bt_solver_opts* o) {
  if (!o) return BT_EINVAL;
  o->tol_fp64 = 1e-12;
  o->tol_inner = 1e-4;
  o->tol_ref = 1e-8;
  o->max_iter = 1000;
  o->max_refine = 6;
  o->check_every = 4;
  o->flags = 0;
  o->rhs_begin = 0;
  o->rhs_end = 0;
  return BT_OK;
}

}  // extern "C"

namespace {

// RHS per lane: the NB right-hand sides of a lane must share one direction
// NB consecutive systems of one lane must share a direction, and with NB > 1
// the RHS count must fill whole tiles of 32 NB columns
int pick_nb(const bt_ctx* ctx, int rb, int Rs) {
  for (int nb : {4, 2}) {
    if (ctx->n_b % nb == 0 && rb % nb == 0 && Rs % (32 * nb) == 0) return nb;
  }
  return 1;
}

}  // namespace

namespace {
// Halo tiles for RHS-per-lane nb (umax from the shared-memory budget) and the
// plane values in halo-entry order.  Sets ctx->halo_ok = false when a row is
// wider than umax (the halo iteration is then not offered).
bt_status ensure_halo(bt_ctx* ctx, int nb, cudaStream_t st) {
  const int umax = halo_umax(nb);
  if (!ctx->halo_attr) {
    halo_prepare();
    resid_df_halo_prepare();
    CKL();
    ctx->halo_attr = true;
  }
  if (ctx->halo_for != ctx->seg_row0 || ctx->halo_umax != umax) {
    HaloTiles t;
    build_halo_tiles(ctx->mesh, ctx->seg_row0, umax, HALO_TMAX, HALO_EMAX, t);
    ctx->halo_for = ctx->seg_row0;
    ctx->halo_umax = umax;
    ctx->halo_ok = !t.too_wide;
    ctx->halo_planes_version = -1;
    if (!ctx->halo_ok) return BT_OK;
    CK(upload(ctx->h_r0, t.r0, st));
    CK(upload(ctx->h_rows, t.rows, st));
    CK(upload(ctx->h_rowe, t.rowe, st));
    CK(upload(ctx->h_rowl, t.rowl, st));
    CK(upload(ctx->h_u0, t.u0, st));
    CK(upload(ctx->h_e0, t.e0, st));
    CK(upload(ctx->h_ucol, t.ucol, st));
    t.lidx.push_back(0);  // padding: the kernels copy local indices in 4-byte words
    t.lidx.push_back(0);
    CK(upload(ctx->h_lidx, t.lidx, st));
    CK(upload(ctx->h_slot, t.slot, st));
    CK(upload(ctx->h_seg0, t.seg_tile0, st));
    CK(cudaStreamSynchronize(st));
  }
  if (ctx->halo_ok && ctx->halo_planes_version != ctx->planes_version) {
    CK(ensure(ctx->h_pkt, ctx->mesh.nnz));
    CK(ensure(ctx->h_mdt, ctx->mesh.nnz));
    launch_gather_tile_planes(ctx->h_slot.p, ctx->mesh.nnz, ctx->d_pk32.p, ctx->d_md32.p, ctx->h_pkt.p,
                              ctx->h_mdt.p, st);
    CK(ensure(ctx->h_dft, 3 * (size_t)ctx->mesh.nnz));
    launch_gather_tile_df(ctx->h_slot.p, ctx->mesh.nnz, ctx->d_pkhi.p, ctx->d_pklo.p, ctx->d_kjmd_hi.p,
                          ctx->d_kjmd_lo.p, ctx->h_dft.p, st);
    CKL();
    ctx->halo_planes_version = ctx->planes_version;
  }
  return BT_OK;
}

HaloArgs halo_args(const bt_ctx* ctx) {
  return HaloArgs{ctx->h_r0.p,   ctx->h_rows.p, ctx->h_rowe.p, ctx->h_rowl.p, ctx->h_u0.p,  ctx->h_e0.p,
                  ctx->h_ucol.p, ctx->h_lidx.p, ctx->h_pkt.p,  ctx->h_mdt.p,  ctx->h_dft.p,  ctx->h_seg0.p,
                  ctx->halo_umax};
}

// Slice tiles of each class (owned rows longest first, FP32 planes in
// tile-entry order) and the plan of tile blocks of each configuration for S
// slices of 32 systems: the configuration's resident blocks per SM times the
// SMs in all, split over the segments in proportion to their tiles, at least
// one each.  A class whose tiles a row does not fit (ok = false) is not
// offered.
bt_status ensure_slice(bt_ctx* ctx, int S, cudaStream_t st) {
  if (!ctx->slice_attr) {
    slice_prepare();
    CKL();
    ctx->slice_attr = true;
  }
  for (int cls = 0; cls < SLICE_NCLS; ++cls) {
    auto& T = ctx->slice_t[cls];
    int c0 = 0;
    while (SLICE_CONF[c0].cls != cls) ++c0;
    const SliceConf& sc = SLICE_CONF[c0];
    if (T.made_for != ctx->seg_row0) {
      HaloTiles t;
      for (int c = 0; c < SLICE_NCONF; ++c)
        if (SLICE_CONF[c].cls == cls) ctx->slice_plan[c].S = 0;
      build_halo_tiles(ctx->mesh, ctx->seg_row0, sc.umax, sc.tmax, sc.emax, t, true);
      T.made_for = ctx->seg_row0;
      T.ok = !t.too_wide;
      T.planes_version = -1;
      if (!T.ok) continue;
      CK(upload(T.r0, t.r0, st));
      CK(upload(T.rows, t.rows, st));
      CK(upload(T.rowe, t.rowe, st));
      t.rowl.push_back(0);  // padding: the kernel copies local row indices in 4-byte words
      t.rowl.push_back(0);
      CK(upload(T.rowl, t.rowl, st));
      CK(upload(T.u0, t.u0, st));
      CK(upload(T.e0, t.e0, st));
      CK(upload(T.ucol, t.ucol, st));
      t.lidx.push_back(0);  // padding: the kernel copies local indices in 4-byte words
      t.lidx.push_back(0);
      CK(upload(T.lidx, t.lidx, st));
      CK(upload(T.slot, t.slot, st));
      CK(upload(T.seg0, t.seg_tile0, st));
      T.seg_tile0 = t.seg_tile0;
      CK(cudaStreamSynchronize(st));
    }
    if (!T.ok) continue;
    if (T.planes_version != ctx->planes_version) {
      CK(ensure(T.pkt, ctx->mesh.nnz));
      CK(ensure(T.mdt, ctx->mesh.nnz));
      launch_gather_tile_planes(T.slot.p, ctx->mesh.nnz, ctx->d_pk32.p, ctx->d_md32.p, T.pkt.p, T.mdt.p, st);
      CKL();
      T.planes_version = ctx->planes_version;
    }
  }
  for (int c = 0; c < SLICE_NCONF; ++c) {
    const auto& T = ctx->slice_t[SLICE_CONF[c].cls];
    auto& pl = ctx->slice_plan[c];
    if (!T.ok || pl.S == S) continue;
    const int G = ctx->G;
    const auto& t0 = T.seg_tile0;
    const int64_t nT = std::max<int64_t>(1, t0[G] - t0[0]);
    const int target = std::max(1, ctx->sms * SLICE_CONF[c].blocks / S);  // resident blocks
    std::vector<int> blk_seg, blk0(G + 1, 0);
    for (int g = 0; g < G; ++g) {
      const int64_t Tg = t0[g + 1] - t0[g];
      int64_t nbg = (int64_t)std::llround((double)target * Tg / (double)nT);
      nbg = std::max<int64_t>(1, std::min<int64_t>(nbg, std::max<int64_t>(1, Tg)));
      blk0[g + 1] = blk0[g] + (int)nbg;
      for (int64_t k = 0; k < nbg; ++k) blk_seg.push_back(g);
    }
    CK(upload(pl.blk_seg, blk_seg, st));
    CK(upload(pl.blk0, blk0, st));
    CK(cudaStreamSynchronize(st));
    pl.nblk = blk0[G];
    pl.S = S;
  }
  return BT_OK;
}

// Krylov variants 2..5 are the slice-tiled iteration in configuration
// variant - 2; whether that configuration's tiles exist
int slice_cfg(int variant) { return variant - 2; }
bool slice_cfg_ok(const bt_ctx* ctx, int cfg) { return ctx->slice_t[SLICE_CONF[cfg].cls].ok; }

HaloArgs slice_args(const bt_ctx* ctx, int cfg) {
  const auto& T = ctx->slice_t[SLICE_CONF[cfg].cls];
  return HaloArgs{T.r0.p,   T.rows.p, T.rowe.p, T.rowl.p, T.u0.p,   T.e0.p,  T.ucol.p,
                  T.lidx.p, T.pkt.p,  T.mdt.p,  nullptr,  T.seg0.p, SLICE_CONF[cfg].umax};
}
// the x/p update of the slice iteration keeps a counter of its own (it only
// uses the last-block ticket)
RedScratch rs_xp(const bt_ctx* ctx) { return RedScratch{ctx->red_part.p, ctx->red_counter.p + 10}; }
SegPlan slice_plan(const bt_ctx* ctx, int cfg) {
  const auto& pl = ctx->slice_plan[cfg];
  return SegPlan{pl.blk_seg.p, pl.blk0.p, ctx->d_row0.p, ctx->G, pl.nblk};
}

// Autotuner: time one Krylov iteration of each variant on the real pattern
// and RHS count (CUDA events, 3 iterations after a warm-up) and keep the
// faster, cached per (RHS, RHS per lane, segments):
//   0: row SpMM + vector update + p update
//   1: halo-staged apply + z update (when the halo tiles exist and allow_halo)
// The Krylov state is primed with benign scalars (nothing converges while
// timing); the Krylov init of the first solve re-initialises all of it.
bt_status autotune_spmm(bt_ctx* ctx, const OpArgs& op, const VecArgs& va, const KrylovState& ks,
                        const RefineState& rf, RedScratch rs, RedScratch rs2, int conj, int nb, int SY, int Rs, int G,
                        bool allow_halo, bool allow_slice, bool df, int* variant, bool* resid_halo) {
  bt_ctx::Tuned* hit = nullptr;
  for (auto& t : ctx->tuned)
    if (t.R == Rs && t.nb == nb && t.G == G) hit = &t;
  const bool halo = allow_halo && ctx->halo_ok;
  bool slice_ok[SLICE_NCONF], slice_untimed = false;
  for (int c = 0; c < SLICE_NCONF; ++c) {
    slice_ok[c] = allow_slice && slice_cfg_ok(ctx, c);
    if (slice_ok[c] && hit && hit->ms[2 + c] == 0) slice_untimed = true;
  }
  if (!hit || (halo && hit->ms[1] == 0) || slice_untimed || (halo && df && hit->ms_resid[1] == 0)) {
    cudaStream_t st = ctx->stream;
    const size_t NE = (size_t)op.n * op.Rp;
    std::vector<double> one(2 * (size_t)SY), small(2 * (size_t)SY), half(2 * (size_t)SY), big(SY, 1e300);
    for (int s2 = 0; s2 < SY; ++s2) {
      one[2 * s2] = 1.0;
      small[2 * s2] = 0.1;
      half[2 * s2] = 0.5;
    }
    auto prime = [&]() -> bt_status {
      launch_set_int(ks.active, 1, SY, st);
      launch_set_int(ks.n_active, SY, 1, st);
      launch_set_int(ks.iter, 0, SY, st);
      launch_set_int(ks.it_best, 0, SY, st);
      if (ks.pend) launch_set_int(ks.pend, 1, SY, st);
      if (ks.par) launch_set_int(ks.par, 0, 1, st);
      CK(cudaMemcpyAsync(ks.rho, one.data(), one.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(ks.alpha, small.data(), small.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(ks.beta, half.data(), half.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemsetAsync(ks.tol2, 0, SY * sizeof(double), st));
      CK(cudaMemcpyAsync(ks.rr_best, big.data(), big.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      return BT_OK;
    };
    // every variant starts from the same vectors (a variant timed after
    // another must not inherit iterates that may have converged or overflowed)
    auto reset_vectors = [&]() -> bt_status {
      for (float2* b : {ctx->x32.p, ctx->r32.p, ctx->p32.p, ctx->q32.p, ctx->p32b.p})
        if (b) CK(cudaMemsetAsync(b, 0x3e, NE * sizeof(float2), st));
      return BT_OK;
    };
    auto iter = [&](int v) {
      if (v >= 2) {
        launch_spmm_slice(op, slice_args(ctx, slice_cfg(v)), slice_plan(ctx, slice_cfg(v)), ctx->p32.p, ctx->q32.p,
                          ks, rs, conj, nb, slice_cfg(v), st);
        launch_slice_r(op, va, ctx->r32.p, ctx->q32.p, ks, rs2, conj, st);
        launch_slice_xp(op, va, ctx->x32.p, ctx->p32.p, ctx->r32.p, ks, rs_xp(ctx), st);
      } else if (v == 1) {
        launch_spmm_halo(op, halo_args(ctx), ctx->r32.p, ctx->p32.p, ctx->p32b.p, ctx->x32.p, ctx->q32.p, ks, rs,
                         conj, nb, st);
        launch_krylov_update_z(op, va, ctx->r32.p, ctx->q32.p, ks, rs2, conj, st);
      } else {
        launch_spmm_krylov_f32(op, ctx->p32.p, ctx->q32.p, ks, rs, conj, nb, ctx->sms, st);
        launch_krylov_update_f32(op, va, ctx->x32.p, ctx->r32.p, ctx->p32.p, ctx->q32.p, ks, rs2, conj, ctx->sms,
                                 st);
        launch_krylov_p_f32(op, va, ctx->r32.p, ctx->p32.p, ks, ctx->sms, st);
      }
    };
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    bt_ctx::Tuned tu{Rs, nb, G, 0, {}, {0, 0}};
    for (int v = 0; v < 2 + SLICE_NCONF; ++v) {
      if ((v == 1 && !halo) || (v >= 2 && !slice_ok[slice_cfg(v)])) continue;
      if (bt_status e = reset_vectors()) return e;
      if (bt_status e = prime()) return e;
      iter(v);  // warm-up
      CK(cudaEventRecord(e0, st));
      for (int k = 0; k < 3; ++k) iter(v);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      tu.ms[v] = ms / 3;
    }
    // the correction residual (double-float): row kernel vs halo tiles, one
    // launch at a time with the refinement state primed before each (a launch
    // may retire systems)
    if (halo && df) {
      std::vector<double> ones(SY, 1.0), huge(SY, 1e300);
      for (float4* b : {ctx->udf.p, ctx->rdf.p})
        if (b) CK(cudaMemsetAsync(b, 0x3e, NE * sizeof(float4), st));
      for (int v = 0; v < 2; ++v) {
        float tot = 0;
        for (int k = 0; k < 3; ++k) {
          launch_set_int(rf.active, 1, SY, st);
          launch_set_int(rf.n_active, SY, 1, st);
          CK(cudaMemcpyAsync(rf.scale, ones.data(), SY * sizeof(double), cudaMemcpyHostToDevice, st));
          CK(cudaMemcpyAsync(rf.r0n2, ones.data(), SY * sizeof(double), cudaMemcpyHostToDevice, st));
          CK(cudaMemcpyAsync(rf.rk2, huge.data(), SY * sizeof(double), cudaMemcpyHostToDevice, st));
          CK(cudaEventRecord(e0, st));
          if (v == 1)
            launch_resid_sub_df_halo(op, halo_args(ctx), ctx->x32.p, ctx->udf.p, ctx->rdf.p, rf, rs, nb, st);
          else launch_resid_sub_df(op, ctx->x32.p, ctx->udf.p, ctx->rdf.p, rf, rs, nb, ctx->sms, st);
          CK(cudaEventRecord(e1, st));
          CK(cudaEventSynchronize(e1));
          float ms = 0;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (k > 0) tot += ms;  // the first launch is the warm-up
        }
        tu.ms_resid[v] = tot / 2;
      }
      CK(cudaMemsetAsync(rf.err, 0, SY * sizeof(double), st));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CKL();
    CK(cudaMemsetAsync(ctx->ks_status.p, 0, SY * sizeof(int), st));
    if (hit) *hit = tu;
    else ctx->tuned.push_back(tu);
    hit = hit ? hit : &ctx->tuned.back();
  }
  int best = 0;
  for (int v = 1; v < 2 + SLICE_NCONF; ++v) {
    const bool avail = v == 1 ? halo : slice_ok[slice_cfg(v)];
    if (avail && hit->ms[v] > 0 && hit->ms[v] < hit->ms[best]) best = v;
  }
  *variant = best;
  *resid_halo = halo && df && hit->ms_resid[1] > 0 && hit->ms_resid[1] < hit->ms_resid[0];
  hit->variant = *variant;
  hit->resid_halo = *resid_halo;
  return BT_OK;
}

// z = P_c r for the polynomial systems of the current inner solve (Horner,
// ping-pong zA/zB, ending in zA), z = D^-1 r for Jacobi systems
bt_status apply_poly(bt_ctx* ctx, const OpArgs& op, const VecArgs& va, const KrylovState& ks, cudaStream_t st) {
  float2* bufs[2] = {ctx->zA.p, ctx->zB.p};
  for (int j = MLP_OUT - 1, w = 0; j >= 0; --j, w ^= 1) {
    launch_horner(op, va, bufs[w ^ 1], ctx->r32.p, bufs[w], ctx->d_coef9.p, j, ks.active, ctx->pmode.p,
                  ks.n_active, ctx->sms, st);
  }
  ctx->st_horner += MLP_OUT;
  CKL();
  return BT_OK;
}
}  // namespace

namespace {
// training-data collection during a run (bt_collect_precond_data)
struct CollectSpec {
  std::vector<int> steps;  // 1-based, ascending
  float* feat;
  double* G;
  double* h;
};
}  // namespace

// At a sampled step: v_0 = D^-1 r (the p of the fresh Krylov init),
// v_{j+1} = D^-1 L v_j (Horner kernel with zero coefficients), then the Gram
// data of every RHS; samples without a step residual get zero G.
static bt_status collect_samples(bt_ctx* ctx, OpArgs op, const VecArgs& va, const KrylovState& ks, int Rs, int Rp,
                                 size_t NE, double fq, const CollectSpec* col, size_t k) {
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ctx->d_coef9.p, 0, 9 * (size_t)Rs * sizeof(double), st));
  launch_set_int(ctx->pmode.p, 1, Rs, st);
  CK(cudaMemcpyAsync(ctx->Vbuf.p, ctx->p32.p, NE * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  for (int j = 0; j < 9; ++j)
    launch_horner(op, va, ctx->Vbuf.p + (size_t)j * NE, ctx->r32.p, ctx->Vbuf.p + (size_t)(j + 1) * NE,
                  ctx->d_coef9.p, 0, ks.active, ctx->pmode.p, ks.n_active, ctx->sms, st);
  launch_gram(op, va, ctx->r32.p, ctx->Vbuf.p, NE, ctx->gram_part.p, ctx->red_counter.p + 7, ctx->gram_out.p,
              ctx->sms, st);
  CKL();
  std::vector<double> g((size_t)Rs * 55);
  std::vector<int> act(Rs);
  CK(cudaMemcpyAsync(g.data(), ctx->gram_out.p, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(act.data(), ks.active, Rs * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int s = 0; s < Rs; ++s) {
    const size_t o = k * Rs + s;
    float* f = col->feat + 5 * o;
    f[0] = (float)ctx->dt;
    f[1] = (float)(ctx->q_rhs[s] * std::fabs(fq));
    f[2] = (float)ctx->feat_D;
    f[3] = (float)ctx->feat_kappa;
    f[4] = (float)ctx->feat_h;
    double* G = col->G + 81 * o;
    double* h = col->h + 9 * o;
    const double* gs = &g[(size_t)s * 55];
    const double rr = gs[54];
    const bool ok = act[s] && rr > 0;
    int q = 0;
    for (int a2 = 0; a2 < 9; ++a2)
      for (int b2 = a2; b2 < 9; ++b2, ++q) G[9 * a2 + b2] = G[9 * b2 + a2] = ok ? gs[q] / rr : 0.0;
    for (int a2 = 0; a2 < 9; ++a2) h[a2] = ok ? gs[45 + a2] / rr : 0.0;
  }
  return BT_OK;
}

// Mixed mode with the time step captured once as a CUDA graph: refinement
// loop and inner Krylov loop are nested WHILE conditional nodes whose
// conditions device kernels set from the convergence counters, the step and
// its coefficients come from a device counter, so the host only launches the
// graph once per step.  Returns BT_ECUDA (and leaves the state untouched, as
// nothing ran) when the graph cannot be built; the caller then drives the same
// kernels from the host.
struct GraphRun {
  int variant;
  bool resid_halo;
  bool weak;
  WeakArgs wa;
  OpArgs op;
  VecArgs va;
  KrylovState ks;
  RefineState rf;
  bool df;
  int conj, nb, N;
  double tol_inner;
};

static bt_status run_graph(bt_ctx* ctx, const GraphRun& g, const bt_solver_opts& o, int Rs, int G,
                           int64_t* iters, int64_t* passes) {
  // the graph is captured on private streams (capture runs nothing, and the
  // legacy default stream cannot be captured) and launched on the context's stream
  cudaStream_t run_st = ctx->stream;
  for (auto& s : ctx->cap_stream)
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BT_ECUDA;
  cudaStream_t c0 = ctx->cap_stream[3], cs = ctx->cap_stream[2], c2 = ctx->cap_stream[0], c3 = ctx->cap_stream[1];
  if (ensure(ctx->d_ctl, 8) != cudaSuccess) return BT_ECUDA;
  const int h0[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  if (cudaMemcpyAsync(ctx->d_ctl.p, h0, sizeof(h0), cudaMemcpyHostToDevice, run_st) != cudaSuccess) return BT_ECUDA;
  if (cudaStreamSynchronize(run_st) != cudaSuccess) return BT_ECUDA;
  GraphCtl gc{ctx->d_ctl.p, g.ks.n_active, ctx->d_seg_N.p, Rs, G, o.max_iter, o.max_refine, g.N};
  OpArgs op0 = g.op, opL = g.op;
  op0.coef = opL.coef = ctx->d_coef.p;
  op0.step = opL.step = ctx->d_ctl.p;
  op0.sel = 0;
  opL.sel = 1;
  auto rs_at = [&](int c) { return RedScratch{ctx->red_part.p, ctx->red_counter.p + c}; };
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = true;
  std::string why;
  int site = 0;
  auto E = [&](cudaError_t e) {
    ++site;
    if (e != cudaSuccess && ok) why = "site " + std::to_string(site) + ": " + cudaGetErrorString(e);
    if (e != cudaSuccess) ok = false;
    return e == cudaSuccess;
  };
  auto while_node = [&](cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg;
    const cudaGraphNode_t* deps;
    size_t nd = 0;
    if (!E(cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, &deps, nullptr, &nd))) return;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (!E(cudaGraphAddNode(&node, capg, deps, nullptr, nd, &p))) return;
    *body = p.conditional.phGraph_out[0];
    E(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  };
  auto capg_of = [&](cudaStream_t s) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg = nullptr;
    E(cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, nullptr, nullptr, nullptr));
    return capg;
  };
  // top level: WHILE (steps left) { one time step }
  cudaGraphConditionalHandle hS{};
  cudaGraph_t bodyS = nullptr;
  if (E(cudaStreamBeginCapture(c0, cudaStreamCaptureModeThreadLocal))) {
    if (E(cudaGraphConditionalHandleCreate(&hS, capg_of(c0), 0, 0))) {
      launch_graph_cond(gc, 4, hS, c0);
      while_node(c0, hS, &bodyS);
    }
  }
  if (ok && E(cudaStreamBeginCaptureToGraph(cs, bodyS, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal))) {
    launch_graph_step_begin(gc, ctx->rf_active.p, cs);
    if (g.df && g.resid_halo && resid_df_halo_available(g.nb, 0))
      launch_resid0_df_halo(op0, halo_args(ctx), ctx->udf.p, ctx->rdf.p, g.rf, rs_at(0), g.nb, cs);
    else if (g.df) launch_resid0_df(op0, ctx->udf.p, ctx->rdf.p, g.rf, rs_at(0), g.nb, ctx->sms, cs);
    else launch_resid0(op0, ctx->u64.p, ctx->r64.p, g.rf, rs_at(0), g.nb, ctx->sms, cs);
    if (g.weak) {
      WeakArgs wg = g.wa;
      wg.step_dev = ctx->d_ctl.p;  // ctl[0]: the 1-based step number
      const void* uu = g.df ? (const void*)ctx->udf.p : (const void*)ctx->u64.p;
      void* rr = g.df ? (void*)ctx->rdf.p : (void*)ctx->r64.p;
      launch_weak_coupling(wg, g.va, op0, uu, rr, g.df, cs);
      launch_resid0_renorm(g.va, uu, rr, g.rf, rs_at(8), g.df, cs);
    }
    cudaGraphConditionalHandle hR{}, hI{};
    cudaGraph_t bodyR = nullptr, bodyI = nullptr;
    cudaGraph_t top = capg_of(cs);
    if (ok) E(cudaGraphConditionalHandleCreate(&hR, top, 0, 0));
    if (ok) launch_graph_cond(gc, 0, hR, cs);
    if (ok) while_node(cs, hR, &bodyR);
    if (ok && E(cudaStreamBeginCaptureToGraph(c2, bodyR, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal))) {
      if (g.variant == 1)
        launch_krylov_init_z(opL, g.va, g.df ? (const void*)ctx->rdf.p : (const void*)ctx->r64.p, g.df,
                             ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p, g.ks, g.tol_inner, rs_at(1),
                             g.conj, c2);
      else if (g.variant >= 2)
        launch_slice_init(opL, g.va, g.df ? (const void*)ctx->rdf.p : (const void*)ctx->r64.p, g.df,
                          ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p, ctx->p32.p, g.ks, g.tol_inner,
                          rs_at(1), g.conj, c2);
      else if (g.df)
        launch_krylov_init_f32_df(opL, g.va, ctx->rdf.p, ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p,
                                  ctx->p32.p, g.ks, g.tol_inner, rs_at(1), g.conj, ctx->sms, c2);
      else
        launch_krylov_init_f32(opL, g.va, ctx->r64.p, ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p,
                               ctx->p32.p, g.ks, g.tol_inner, rs_at(1), g.conj, ctx->sms, c2);
      if (E(cudaGraphConditionalHandleCreate(&hI, bodyR, 0, 0))) {
        launch_graph_cond(gc, 2, hI, c2);
        while_node(c2, hI, &bodyI);
        if (ok && E(cudaStreamBeginCaptureToGraph(c3, bodyI, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal))) {
          if (g.variant == 1) {
            launch_spmm_halo(opL, halo_args(ctx), ctx->r32.p, ctx->p32.p, ctx->p32b.p, ctx->x32.p, ctx->q32.p, g.ks,
                             rs_at(2), g.conj, g.nb, c3);
            launch_krylov_update_z(opL, g.va, ctx->r32.p, ctx->q32.p, g.ks, rs_at(3), g.conj, c3);
          } else if (g.variant >= 2) {
            launch_spmm_slice(opL, slice_args(ctx, slice_cfg(g.variant)), slice_plan(ctx, slice_cfg(g.variant)),
                              ctx->p32.p, ctx->q32.p, g.ks, rs_at(2), g.conj, g.nb, slice_cfg(g.variant), c3);
            launch_slice_r(opL, g.va, ctx->r32.p, ctx->q32.p, g.ks, rs_at(3), g.conj, c3);
            launch_slice_xp(opL, g.va, ctx->x32.p, ctx->p32.p, ctx->r32.p, g.ks, rs_xp(ctx), c3);
          } else {
            launch_spmm_krylov_f32(opL, ctx->p32.p, ctx->q32.p, g.ks, rs_at(2), g.conj, g.nb, ctx->sms, c3);
            launch_krylov_update_f32(opL, g.va, ctx->x32.p, ctx->r32.p, ctx->p32.p, ctx->q32.p, g.ks, rs_at(3),
                                     g.conj, ctx->sms, c3);
            launch_krylov_p_f32(opL, g.va, ctx->r32.p, ctx->p32.p, g.ks, ctx->sms, c3);
          }
          launch_graph_cond(gc, 3, hI, c3);
          E(cudaGetLastError());
          cudaGraph_t tmp;
          E(cudaStreamEndCapture(c3, &tmp));
        }
      }
      if (g.variant == 1) launch_flush_x(g.va, ctx->x32.p, ctx->p32.p, ctx->p32b.p, g.ks, c2);
      if (g.df && g.resid_halo)
        launch_resid_sub_df_halo(opL, halo_args(ctx), ctx->x32.p, ctx->udf.p, ctx->rdf.p, g.rf, rs_at(4), g.nb, c2);
      else if (g.df) launch_resid_sub_df(opL, ctx->x32.p, ctx->udf.p, ctx->rdf.p, g.rf, rs_at(4), g.nb, ctx->sms, c2);
      else launch_resid_sub(opL, ctx->x32.p, ctx->u64.p, ctx->r64.p, g.rf, rs_at(4), g.nb, ctx->sms, c2);
      launch_graph_cond(gc, 1, hR, c2);
      E(cudaGetLastError());
      cudaGraph_t tmp;
      E(cudaStreamEndCapture(c2, &tmp));
    }
    launch_mark_ref_left(g.rf, g.ks, Rs * G, cs);
    launch_graph_step_end(gc, cs);
    launch_graph_cond(gc, 4, hS, cs);
    E(cudaGetLastError());
    cudaGraph_t tmp = nullptr;
    E(cudaStreamEndCapture(cs, &tmp));
  }
  {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c0, &cst);
    if (cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t tmp = nullptr;
      const bool was_ok = ok;
      const cudaError_t ee = cudaStreamEndCapture(c0, &tmp);
      if (ee != cudaSuccess && was_ok) why = std::string("end capture: ") + cudaGetErrorString(ee);
      if (ee != cudaSuccess) ok = false;
      graph = tmp;
    }
  }
  if (ok && graph) E(cudaGraphInstantiate(&exec, graph, 0));
  if (!ok || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    // not an error of the run: the caller drives the same kernels from the host
    ctx->err = "run graph unavailable (" + why + "); host-driven launches used";
    return BT_ECUDA;
  }
  ok = cudaGraphLaunch(exec, run_st) == cudaSuccess;  // the whole simulation
  int hc[8] = {0};
  if (ok) ok = cudaMemcpyAsync(hc, ctx->d_ctl.p, sizeof(hc), cudaMemcpyDeviceToHost, run_st) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(run_st) == cudaSuccess;
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (!ok) return fail(ctx, BT_ECUDA, std::string("bt_run: graph launch failed: ") + cudaGetErrorString(cudaGetLastError()));
  *iters = hc[3];
  *passes = hc[4] + 0;
  return BT_OK;
}

static bt_status run_impl(bt_ctx* ctx, int mode, const bt_solver_opts* opts_in, const CollectSpec* col) {
  if (!ctx) return BT_EINVAL;
  if (!need_gpu(ctx)) return fail(ctx, BT_ENODEV, "bt_run: host-only context");
  if (!ctx->assembled || !ctx->have_seq || ctx->R == 0)
    return fail(ctx, BT_ESTATE, "bt_run: need mesh, assembly, sequence and gradients");
  if (mode != BT_MODE_PLAIN_FP64 && mode != BT_MODE_MIXED && mode != BT_MODE_LEARNED)
    return fail(ctx, BT_EINVAL, "bt_run: unknown mode");
  if (mode == BT_MODE_LEARNED && !ctx->have_precond && !ctx->have_fixed_poly)
    return fail(ctx, BT_ESTATE, "bt_run: BT_MODE_LEARNED needs a trained, loaded or fixed preconditioner");
  const bool learned = mode == BT_MODE_LEARNED;
  bt_solver_opts o;
  bt_default_opts(&o);
  if (opts_in) o = *opts_in;
  int rb = o.rhs_begin, re = o.rhs_end;
  if (rb == 0 && re == 0) re = ctx->R;
  if (rb < 0 || re > ctx->R || rb >= re) return fail(ctx, BT_EINVAL, "bt_run: bad RHS range");
  const int G = ctx->G;
  if (G > 1 && (rb != 0 || re != ctx->R)) return fail(ctx, BT_EINVAL, "bt_run: RHS ranges need a single segment");
  if (G > 1 && (learned || col)) return fail(ctx, BT_EINVAL, "bt_run: learned mode and data collection need a single segment");
  if (G > 1 && ctx->weak_axes) return fail(ctx, BT_EINVAL, "bt_run: the weak periodic box needs a single segment");
  if (o.max_iter < 1 || o.max_refine < 1 || o.check_every < 1 || !(o.tol_fp64 > 0) || !(o.tol_inner > 0) ||
      !(o.tol_ref > 0))
    return fail(ctx, BT_EINVAL, "bt_run: bad solver options");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ctx->last_kind = 0;
  const int Rs = re - rb;
  const int nb = pick_nb(ctx, rb, Rs);
  const int Rp = ((Rs + nb - 1) / nb) * nb;
  const int64_t n = ctx->mesh.n_dof;
  const size_t NE = (size_t)n * Rp;
  const bool plain = mode == BT_MODE_PLAIN_FP64;
  const bool df = !plain && !(o.flags & BT_OPT_RESID_FP64);
  const bool prof = (o.flags & BT_OPT_PROFILE) != 0;
  const bool narrow = plain && Rs <= 4 && G == 1;  // lanes over nonzeros for the per-direction FP64 solve
  const int SY = G * Rs;                            // systems: G segments x Rs right-hand sides
  const int conj = ctx->transformed ? 1 : 0;  // CG (Hermitian) vs COCG (complex symmetric)

  // per-run device buffers
  CK(ensure(ctx->d_q, SY));
  CK(ensure(ctx->d_qhat, 3 * (size_t)SY));
  CK(cudaMemcpyAsync(ctx->d_q.p, ctx->q_rhs.data() + rb, SY * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_qhat.p, ctx->qhat_rhs.data() + 3 * rb, 3 * SY * sizeof(double), cudaMemcpyHostToDevice,
                     st));
  // block plan: blocks in proportion to segment rows, each block in one segment
  {
    const int target = ctx->sms * REDUCE_BLOCKS_PER_SM;
    std::vector<int> blk_seg, blk0(G + 1, 0);
    for (int g = 0; g < G; ++g) {
      const int64_t rows = ctx->seg_row0[g + 1] - ctx->seg_row0[g];
      const int64_t chunks = (rows + ROW_CHUNK - 1) / ROW_CHUNK;
      int64_t nbg = (int64_t)std::llround((double)target * rows / (double)n);
      nbg = std::max<int64_t>(1, std::min(nbg, chunks));
      blk0[g + 1] = blk0[g] + (int)nbg;
      for (int64_t k = 0; k < nbg; ++k) blk_seg.push_back(g);
    }
    ctx->nblk = blk0[G];
    CK(upload(ctx->d_blk_seg, blk_seg, st));
    CK(upload(ctx->d_blk0, blk0, st));
    CK(upload(ctx->d_row0, ctx->seg_row0, st));
    CK(upload(ctx->d_seg_N, ctx->seg_N, st));
  }
  const SegPlan sp{ctx->d_blk_seg.p, ctx->d_blk0.p, ctx->d_row0.p, G, ctx->nblk};
  if (plain) {
    CK(ensure(ctx->u64, NE));
    CK(ensure(ctx->r64, NE));
    CK(ensure(ctx->x64, NE));
    CK(ensure(ctx->rk64, NE));
    CK(ensure(ctx->p64, NE));
    CK(ensure(ctx->q64, NE));
  } else {
    if (df) {
      CK(ensure(ctx->udf, NE));
      CK(ensure(ctx->rdf, NE));
    } else {
      CK(ensure(ctx->u64, NE));
      CK(ensure(ctx->r64, NE));
    }
    CK(ensure(ctx->x32, NE));
    CK(ensure(ctx->r32, NE));
    CK(ensure(ctx->p32, NE));
    CK(ensure(ctx->q32, NE));
    if (!learned && !col) CK(ensure(ctx->p32b, NE));
  }
  CK(ensure(ctx->ks_pend, SY));
  CK(ensure(ctx->ks_par, 1));
  CK(ensure(ctx->d_sys_iter, 1 + (size_t)G));
  CK(ensure(ctx->ks_rho, 2 * (size_t)SY));
  CK(ensure(ctx->ks_alpha, 2 * (size_t)SY));
  CK(ensure(ctx->ks_beta, 2 * (size_t)SY));
  CK(ensure(ctx->ks_rr0, SY));
  CK(ensure(ctx->ks_rr, SY));
  CK(ensure(ctx->ks_tol2, SY));
  CK(ensure(ctx->ks_iter, SY));
  CK(ensure(ctx->ks_active, SY));
  CK(ensure(ctx->ks_status, SY));
  CK(ensure(ctx->ks_rr_best, SY));
  CK(ensure(ctx->ks_it_best, SY));
  CK(ensure(ctx->n_active, 4));
  CK(ensure(ctx->rf_r0n2, SY));
  CK(ensure(ctx->rf_rk2, SY));
  CK(ensure(ctx->rf_scale, SY));
  CK(ensure(ctx->rf_err, SY));
  CK(ensure(ctx->rf_active, SY));
  CK(ensure(ctx->d_S, 2 * (size_t)SY));
  if (learned || col) {
    CK(ensure(ctx->zA, NE));
    CK(ensure(ctx->zB, NE));
    CK(ensure(ctx->pmode, SY));
    CK(ensure(ctx->d_feat, 5 * (size_t)Rs));
    CK(ensure(ctx->d_coef9, 9 * (size_t)Rs));
  }
  if (col) {
    CK(ensure(ctx->Vbuf, 10 * NE));
    CK(ensure(ctx->gram_part, (size_t)(2 * ctx->sms + 8) * Rp * 55));
    CK(ensure(ctx->gram_out, (size_t)Rs * 55));
  }
  const size_t max_blocks = (size_t)std::max(ctx->sms * REDUCE_BLOCKS_PER_SM, ctx->nblk) + 64;
  CK(ensure(ctx->red_part, max_blocks * Rp * 6));  // up to three complex partials per (block, RHS)
  // coefficient table: per step, [0] = r_0 operator (R_n - L_n), [1] = L_n
  // coefficient table [step][0 = r_0 operator (R_n - L_n), 1 = L_n][segment]
  const int N = ctx->n_steps;
  std::vector<OpCoef> coefs(2 * (size_t)N * G, OpCoef{0.0, 0.0, 0.0});
  const double dt = ctx->dt, th = ctx->theta;
  for (int s = 1; s <= N; ++s)
    for (int g = 0; g < G; ++g) {
      if (s > ctx->seg_N[g]) continue;  // segment finished: frozen
      OpCoef c0, c1;
      if (!ctx->transformed) {
        const double fb = ctx->seg_fbar[g][s - 1];
        c0 = {-dt, 0.0, -dt * fb};
        c1 = {1.0, 0.0, th * dt * fb};
      } else {
        const double Fn = ctx->seg_F[g][s], Fp = ctx->seg_F[g][s - 1];
        c0 = {-dt, -dt * ((1 - th) * Fp * Fp + th * Fn * Fn), -dt * ((1 - th) * Fp + th * Fn)};
        c1 = {1.0, th * dt * Fn * Fn, th * dt * Fn};
      }
      coefs[(2 * (size_t)(s - 1)) * G + g] = c0;
      coefs[(2 * (size_t)(s - 1) + 1) * G + g] = c1;
    }
  CK(ensure(ctx->d_coef, coefs.size()));
  CK(cudaMemcpyAsync(ctx->d_coef.p, coefs.data(), coefs.size() * sizeof(OpCoef), cudaMemcpyHostToDevice, st));

  OpArgs op{};
  op.rp = ctx->d_rp.p;
  op.col = ctx->d_col.p;
  op.n = n;
  op.pk64 = ctx->d_pk64.p;
  op.p0_64 = ctx->d_KJ.p;
  op.p1_64 = ctx->d_planes.p + 3 * (size_t)ctx->mesh.nnz;  // MD plane
  op.pk32 = ctx->d_pk32.p;
  op.p1_32 = ctx->d_md32.p;
  op.pkhi = ctx->d_pkhi.p;
  op.pklo = ctx->d_pklo.p;
  op.kjmd_hi = ctx->d_kjmd_hi.p;
  op.kjmd_lo = ctx->d_kjmd_lo.p;
  op.q = ctx->d_q.p;
  op.qhat = ctx->d_qhat.p;
  op.R = Rs;
  op.Rp = Rp;
  op.transformed = ctx->transformed;
  op.sp = sp;
  VecArgs va{n, Rs, Rp, nb, sp, ctx->d_diag64.p, ctx->d_diag_md64.p, ctx->d_diag32.p, ctx->d_diag_md32.p};
  KrylovState ks{ctx->ks_rho.p, ctx->ks_alpha.p, ctx->ks_beta.p, ctx->ks_rr0.p, ctx->ks_rr.p, ctx->ks_tol2.p,
                 ctx->ks_iter.p, ctx->ks_active.p, ctx->n_active.p, ctx->ks_status.p, ctx->ks_rr_best.p,
                 ctx->ks_it_best.p, o.max_iter, plain ? 0 : 30, ctx->ks_par.p, ctx->ks_pend.p, ctx->d_sys_iter.p};
  RefineState rf{ctx->rf_r0n2.p, ctx->rf_rk2.p, ctx->rf_scale.p, ctx->rf_err.p, ctx->rf_active.p,
                 ctx->n_active.p + 1, o.tol_ref * o.tol_ref, 0.0, ctx->ks_status.p};
  const double feps = 1e-14 * ctx->wmax;
  rf.floor_c2 = feps * feps;
  auto rs_at = [&](int c) { return RedScratch{ctx->red_part.p, ctx->red_counter.p + c}; };
  // weak pseudo-periodic box: partner-face coupling rows and F(t_n)
  const bool weak = ctx->weak_axes != 0;
  WeakArgs wa{};
  if (weak) {
    CK(upload(ctx->d_Fstep, ctx->F, st));
    wa = WeakArgs{ctx->d_wrows.p, ctx->d_wptr.p, ctx->d_wcol.p, ctx->d_ww.p, ctx->d_wcode.p,
                  (int64_t)ctx->weak.rows.size(), {ctx->weak.L[0], ctx->weak.L[1], ctx->weak.L[2]},
                  ctx->theta * ctx->dt * ctx->weak_kappa, ctx->d_Fstep.p, nullptr, 0};
  }

  // halo tiles, the tuned Krylov variant for the FP32 inner solves and the
  // tuned double-float residual kernel
  int variant = 0;
  bool resid_halo = false;
  if (!plain) {
    const bool allow_halo = !learned && !col;
    const bool allow_slice = !learned && !col && Rp % 32 == 0;
    if (allow_halo)
      if (bt_status e = ensure_halo(ctx, nb, st)) return e;
    if (allow_slice)
      if (bt_status e = ensure_slice(ctx, Rp / 32, st)) return e;
    OpArgs opt = op;
    opt.coef = ctx->d_coef.p + G;  // step 1, L operator
    if (bt_status e = autotune_spmm(ctx, opt, va, ks, rf, rs_at(2), rs_at(3), conj, nb, SY, Rs, G, allow_halo,
                                    allow_slice, df, &variant, &resid_halo))
      return e;
    if (o.flags & BT_OPT_VARIANT_ROW) variant = 0, resid_halo = false;
    if ((o.flags & BT_OPT_VARIANT_HALO) && allow_halo && ctx->halo_ok) variant = 1, resid_halo = df;
    const int forced = (int)((o.flags >> BT_OPT_SLICE_CONFIG_SHIFT) & 7u) - 1;  // -1: none
    if (allow_slice && (o.flags & BT_OPT_VARIANT_SLICE) && variant < 2) {
      // the fastest slice configuration that was timed
      const auto& tu = ctx->tuned.back();
      for (int c = 0; c < SLICE_NCONF; ++c)
        if (slice_cfg_ok(ctx, c) && tu.ms[2 + c] > 0 && (variant < 2 || tu.ms[2 + c] < tu.ms[variant])) variant = 2 + c;
    }
    if (allow_slice && (o.flags & BT_OPT_SLICE_ONE_STAGE) && slice_cfg_ok(ctx, 1)) variant = 3;
    if (allow_slice && forced >= 0 && forced < SLICE_NCONF && slice_cfg_ok(ctx, forced)) variant = 2 + forced;
    ctx->last_variant = variant;
    ctx->last_resid_halo = resid_halo ? 1 : 0;
  }
  ctx->st_steps = ctx->st_iters = ctx->st_refine = ctx->st_spmm = ctx->st_resid = ctx->st_launches = 0;
  ctx->st_horner = 0;
  ctx->st_spmm_ms = ctx->st_resid_ms = ctx->st_vec_ms = 0;
  ctx->ev_used = 0;
  CK(cudaMemsetAsync(ctx->rf_err.p, 0, SY * sizeof(double), st));
  CK(cudaMemsetAsync(ctx->ks_status.p, 0, SY * sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_sys_iter.p, 0, (1 + (size_t)G) * sizeof(unsigned long long), st));
  const double* rho_dof = ctx->have_rho ? ctx->d_rho_dof.p : nullptr;
  if (df) launch_fill_u_df(va, ctx->udf.p, rho_dof, st);
  else launch_fill_u(va, ctx->u64.p, rho_dof, st);
  CKL();
  int64_t& L = ctx->st_launches;
  L = 1;

  auto read_flag = [&](const int* dptr, int& out) -> bt_status {
    CK(cudaMemcpyAsync(ctx->h_flags, dptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out = ctx->h_flags[0];
    return BT_OK;
  };
  auto timed = [&](int kind, auto&& launch) {
    EventPair* e = prof ? ev_next(ctx, kind) : nullptr;
    if (e) cudaEventRecord(e->a, st);
    launch();
    if (e) cudaEventRecord(e->b, st);
  };

  // production path: the captured time step (mixed mode)
  bool graph_done = false;
  if (!plain && !learned && !col && !prof && !(o.flags & BT_OPT_NO_GRAPH)) {
    GraphRun gr{variant, resid_halo, weak, wa, op, va, ks, rf, df, conj, nb, N, o.tol_inner};
    int64_t gi = 0, gp = 0;
    if (run_graph(ctx, gr, o, Rs, G, &gi, &gp) == BT_OK) {
      graph_done = true;
      ctx->st_steps = N;
      ctx->st_iters = ctx->st_spmm = gi;
      ctx->st_refine = gp;
      ctx->st_resid = N + gp;
      L += variant == 1 ? 5 * (int64_t)N + 6 * gp + 3 * gi : 5 * (int64_t)N + 4 * gp + 4 * gi;
      if (weak) L += 2 * (int64_t)N;
    }
  }
  double last_fq = NAN;
  size_t col_next = 0;
  std::vector<double> fixed_coef;  // host copy of the fixed polynomial per system (alive during the run)
  if (learned && ctx->have_fixed_poly) {
    fixed_coef.resize(9 * (size_t)Rs);
    for (int s = 0; s < Rs; ++s)
      for (int j = 0; j < 9; ++j) fixed_coef[9 * (size_t)s + j] = ctx->fixed_poly[j];
  }
  for (int step = 1; step <= N && !graph_done; ++step) {
    const OpCoef* c_r0 = ctx->d_coef.p + 2 * (size_t)(step - 1) * G;
    const OpCoef* c_L = c_r0 + G;
    // f_bar_n (lab) or F_n (transformed) of this step: the preconditioner feature
    const double fq = ctx->transformed ? ctx->F[step] : ctx->fbar[step - 1];
    const bool collect_now = col && col_next < col->steps.size() && col->steps[col_next] == step;
    if (learned && ctx->have_fixed_poly) {
      if (step == 1) {  // one polynomial for every system, uploaded once per run
        CK(cudaMemcpyAsync(ctx->d_coef9.p, fixed_coef.data(), fixed_coef.size() * sizeof(double),
                           cudaMemcpyHostToDevice, st));
      }
      launch_set_int(ctx->pmode.p, 1, Rs, st);
      L += 1;
    } else if (learned) {
      if (!(fq == last_fq)) {
        launch_features(ctx->d_q.p, Rs, ctx->dt, fq, ctx->feat_D, ctx->feat_kappa, ctx->feat_h, ctx->d_feat.p, st);
        launch_mlp_forward(ctx->pw16.p, ctx->d_feat.p, Rs, ctx->d_coef9.p, st);
        L += 2;
        last_fq = fq;
      }
      launch_set_int(ctx->pmode.p, 1, Rs, st);
      L += 1;
    }
    int live = 0;  // systems of segments that have not finished
    for (int g = 0; g < G; ++g) live += step <= ctx->seg_N[g] ? Rs : 0;
    launch_seg_active(ctx->rf_active.p, Rs, G, step, ctx->d_seg_N.p, st);
    launch_set_int(rf.n_active, live, 1, st);
    L += 3;  // two set kernels and the step-start residual
    op.coef = c_r0;
    timed(1, [&] {
      if (df && resid_halo && resid_df_halo_available(nb, 0))
        launch_resid0_df_halo(op, halo_args(ctx), ctx->udf.p, ctx->rdf.p, rf, rs_at(0), nb, st);
      else if (df) launch_resid0_df(op, ctx->udf.p, ctx->rdf.p, rf, rs_at(0), nb, ctx->sms, st);
      else if (narrow) launch_resid0_narrow(op, ctx->u64.p, ctx->r64.p, rf, rs_at(0), ctx->sms, st);
      else launch_resid0(op, ctx->u64.p, ctx->r64.p, rf, rs_at(0), nb, ctx->sms, st);
    });
    if (weak) {
      wa.step_host = step;
      const void* uu = df ? (const void*)ctx->udf.p : (const void*)ctx->u64.p;
      void* rr = df ? (void*)ctx->rdf.p : (void*)ctx->r64.p;
      launch_weak_coupling(wa, va, op, uu, rr, df, st);
      launch_resid0_renorm(va, uu, rr, rf, rs_at(8), df, st);
      L += 2;
    }
    CKL();
    ctx->st_resid++;
    op.coef = c_L;
    for (int pass = 0; pass < (plain ? 1 : o.max_refine); ++pass) {
      int nref = 0;
      if (bt_status e = read_flag(rf.n_active, nref)) return e;
      if (nref == 0) break;
      ctx->st_refine++;
      L += 2;  // Krylov init and the closing residual / update
      if (plain) {
        launch_krylov_init_f64(op, va, ctx->r64.p, ctx->rf_active.p, ctx->x64.p, ctx->rk64.p, ctx->p64.p, ks,
                               o.tol_fp64, rs_at(1), conj, ctx->sms, st);
      } else if (variant == 1) {
        launch_krylov_init_z(op, va, df ? (const void*)ctx->rdf.p : (const void*)ctx->r64.p, df, ctx->rf_scale.p,
                             ctx->rf_active.p, ctx->x32.p, ctx->r32.p, ks, o.tol_inner, rs_at(1), conj, st);
      } else if (variant >= 2) {
        launch_slice_init(op, va, df ? (const void*)ctx->rdf.p : (const void*)ctx->r64.p, df, ctx->rf_scale.p,
                          ctx->rf_active.p, ctx->x32.p, ctx->r32.p, ctx->p32.p, ks, o.tol_inner, rs_at(1), conj, st);
      } else if (df) {
        launch_krylov_init_f32_df(op, va, ctx->rdf.p, ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p,
                                  ctx->p32.p, ks, o.tol_inner, rs_at(1), conj, ctx->sms, st);
      } else {
        launch_krylov_init_f32(op, va, ctx->r64.p, ctx->rf_scale.p, ctx->rf_active.p, ctx->x32.p, ctx->r32.p,
                               ctx->p32.p, ks, o.tol_inner, rs_at(1), conj, ctx->sms, st);
      }
      CKL();
      if (collect_now && pass == 0) {
        if (bt_status e = collect_samples(ctx, op, va, ks, Rs, Rp, NE, fq, col, col_next)) return e;
        ++col_next;
      }
      if (learned) {
        // z = P_c r (Horner), then rho = <r, z>, p = z for polynomial systems
        if (bt_status e = apply_poly(ctx, op, va, ks, st)) return e;
        launch_precond_dot(va, ctx->r32.p, ctx->zA.p, ks, rs_at(6), ctx->pmode.p, conj, 1, ctx->sms, st);
        launch_krylov_p_f32(op, va, ctx->r32.p, ctx->p32.p, ks, ctx->sms, st, ctx->zA.p, ctx->pmode.p);
        CKL();
        L += 11;
      }
      for (int it = 0; it < o.max_iter; ++it) {
        if (plain) {
          timed(0, [&] {
            if (narrow) launch_spmm_krylov_f64_narrow(op, ctx->p64.p, ctx->q64.p, ks, rs_at(2), conj, ctx->sms, st);
            else launch_spmm_krylov_f64(op, ctx->p64.p, ctx->q64.p, ks, rs_at(2), conj, nb, ctx->sms, st);
          });
          timed(2, [&] {
            launch_krylov_update_f64(op, va, ctx->x64.p, ctx->rk64.p, ctx->p64.p, ctx->q64.p, ks, rs_at(3), conj,
                                     ctx->sms, st);
            launch_krylov_p_f64(op, va, ctx->rk64.p, ctx->p64.p, ks, ctx->sms, st);
          });
        } else if (variant == 1) {
          timed(0, [&] {
            launch_spmm_halo(op, halo_args(ctx), ctx->r32.p, ctx->p32.p, ctx->p32b.p, ctx->x32.p, ctx->q32.p, ks,
                             rs_at(2), conj, nb, st);
          });
          timed(2, [&] { launch_krylov_update_z(op, va, ctx->r32.p, ctx->q32.p, ks, rs_at(3), conj, st); });
          L -= 1;  // two launches per iteration
        } else if (variant >= 2) {
          timed(0, [&] {
            launch_spmm_slice(op, slice_args(ctx, slice_cfg(variant)), slice_plan(ctx, slice_cfg(variant)), ctx->p32.p,
                              ctx->q32.p, ks, rs_at(2), conj, nb, slice_cfg(variant), st);
          });
          timed(2, [&] {
            launch_slice_r(op, va, ctx->r32.p, ctx->q32.p, ks, rs_at(3), conj, st);
            launch_slice_xp(op, va, ctx->x32.p, ctx->p32.p, ctx->r32.p, ks, rs_xp(ctx), st);
          });
        } else {
          timed(0, [&] { launch_spmm_krylov_f32(op, ctx->p32.p, ctx->q32.p, ks, rs_at(2), conj, nb, ctx->sms, st); });
          timed(2, [&] {
            launch_krylov_update_f32(op, va, ctx->x32.p, ctx->r32.p, ctx->p32.p, ctx->q32.p, ks, rs_at(3), conj,
                                     ctx->sms, st, learned ? ctx->pmode.p : nullptr);
            if (!learned) launch_krylov_p_f32(op, va, ctx->r32.p, ctx->p32.p, ks, ctx->sms, st);
          });
          if (learned) {
            if (bt_status e = apply_poly(ctx, op, va, ks, st)) return e;
            launch_precond_dot(va, ctx->r32.p, ctx->zA.p, ks, rs_at(6), ctx->pmode.p, conj, 0, ctx->sms, st);
            launch_krylov_p_f32(op, va, ctx->r32.p, ctx->p32.p, ks, ctx->sms, st, ctx->zA.p, ctx->pmode.p);
            L += 10;
          }
        }
        CKL();
        ctx->st_iters++;
        ctx->st_spmm++;
        L += 3;
        if ((it + 1) % o.check_every == 0) {
          int na = 0;
          if (bt_status e = read_flag(ks.n_active, na)) return e;
          if (na == 0) break;
        }
      }
      if (plain) {
        launch_axpy_u(va, ctx->x64.p, ctx->u64.p, ks, rf, ctx->sms, st);
        launch_finish_step(rf, ks, SY, st);
        L += 1;
      } else {
        if (variant == 1) {
          launch_flush_x(va, ctx->x32.p, ctx->p32.p, ctx->p32b.p, ks, st);
          L += 2;
        }
        timed(1, [&] {
          if (df && resid_halo)
            launch_resid_sub_df_halo(op, halo_args(ctx), ctx->x32.p, ctx->udf.p, ctx->rdf.p, rf, rs_at(4), nb, st);
          else if (df) launch_resid_sub_df(op, ctx->x32.p, ctx->udf.p, ctx->rdf.p, rf, rs_at(4), nb, ctx->sms, st);
          else launch_resid_sub(op, ctx->x32.p, ctx->u64.p, ctx->r64.p, rf, rs_at(4), nb, ctx->sms, st);
        });
        ctx->st_resid++;
      }
      CKL();
    }
    if (!plain) {
      launch_mark_ref_left(rf, ks, SY, st);
      L += 1;
    }
    ctx->st_steps++;
    if (col && col_next == col->steps.size()) break;  // data collection ends after its last listed step
  }
  op.coef = ctx->d_coef.p;
  if (df) launch_signal_df(va, ctx->d_w.p, ctx->udf.p, ctx->d_S.p, rs_at(5), ctx->sms, st);
  else launch_signal(va, ctx->d_w.p, ctx->u64.p, ctx->d_S.p, rs_at(5), ctx->sms, st);
  CKL();
  L += 1;
  std::vector<double> S(2 * (size_t)SY), err(SY);
  std::vector<int> stat(SY), ref_left(SY);
  CK(cudaMemcpyAsync(S.data(), ctx->d_S.p, 2 * SY * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(err.data(), ctx->rf_err.p, SY * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(stat.data(), ctx->ks_status.p, SY * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ref_left.data(), ctx->rf_active.p, SY * sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<unsigned long long> sys_iter(1 + (size_t)G, 0ULL);
  CK(cudaMemcpyAsync(sys_iter.data(), ctx->d_sys_iter.p, sys_iter.size() * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (prof) ev_harvest(ctx);
  ctx->st_sys_iters = (int64_t)sys_iter[0];
  ctx->st_seg_sys_iters.assign(sys_iter.begin() + 1, sys_iter.end());
  bt_status ret = BT_OK;
  for (int s = 0; s < SY; ++s) {
    ctx->S[2 * (rb + s)] = S[2 * s];
    ctx->S[2 * (rb + s) + 1] = S[2 * s + 1];
    ctx->err_est[rb + s] = err[s];
    int stt = stat[s];
    if (!plain && ref_left[s] && stt == BT_OK) stt = BT_ENOCONV;  // refinement cap hit in the last step
    ctx->status[rb + s] = stt;
    if (stt != BT_OK && ret == BT_OK) ret = stt;
  }
  ctx->last_kind = df ? 2 : 1;
  ctx->last_Rp = Rp;
  ctx->last_nb = nb;
  ctx->last_rb = rb;
  ctx->last_Rs = Rs;
  if (ret != BT_OK) ctx->err = "bt_run: some right-hand sides did not converge (see status)";
  return ret;
}

extern "C" bt_status bt_run(bt_ctx* ctx, int mode, const bt_solver_opts* opts) try {
  return run_impl(ctx, mode, opts, nullptr);
} BT_ABI_CATCH(ctx)

extern "C" bt_status bt_collect_precond_data(bt_ctx* ctx, const bt_solver_opts* opts, int32_t n_steps,
                                             const int32_t* steps, float* feat, double* G, double* h) try {
  if (!ctx || n_steps < 1 || !steps || !feat || !G || !h) return fail(ctx, BT_EINVAL, "bt_collect_precond_data: bad arguments");
  if (!ctx->have_seq) return fail(ctx, BT_ESTATE, "bt_collect_precond_data: set sequence and gradients first");
  CollectSpec c;
  c.steps.assign(steps, steps + n_steps);
  for (int i = 0; i < n_steps; ++i)
    if (c.steps[i] < 1 || c.steps[i] > ctx->n_steps || (i && c.steps[i] <= c.steps[i - 1]))
      return fail(ctx, BT_EINVAL, "bt_collect_precond_data: steps must be ascending in [1, n_steps]");
  bt_solver_opts o;
  bt_default_opts(&o);
  if (opts) o = *opts;
  o.rhs_begin = o.rhs_end = 0;
  c.feat = feat;
  c.G = G;
  c.h = h;
  return run_impl(ctx, BT_MODE_MIXED, &o, &c);
} BT_ABI_CATCH(ctx)

extern "C" bt_status bt_get_signals(bt_ctx* ctx, double* S_re_im, double* err_est, int32_t* status) try {
  if (!ctx) return BT_EINVAL;
  if (ctx->R == 0) return fail(ctx, BT_ESTATE, "bt_get_signals: nothing run");
  const size_t SYt = (size_t)ctx->G * ctx->R;
  if (S_re_im) std::memcpy(S_re_im, ctx->S.data(), 2 * SYt * sizeof(double));
  if (err_est) std::memcpy(err_est, ctx->err_est.data(), SYt * sizeof(double));
  if (status)
    for (size_t i = 0; i < SYt; ++i) status[i] = ctx->status[i];
  return BT_OK;
} BT_ABI_CATCH(ctx)

extern "C" bt_status bt_get_state(bt_ctx* ctx, int32_t system, double* u_re_im, int64_t* n_rows) try {
  if (!ctx) return BT_EINVAL;
  if (!need_gpu(ctx)) return fail(ctx, BT_ENODEV, "bt_get_state: host-only context");
  if (ctx->last_kind == 0) return fail(ctx, BT_ESTATE, "bt_get_state: no state (run first)");
  const int G = ctx->G, R = ctx->R;
  int g = 0, r = 0;
  if (G > 1) {
    if (system < 0 || system >= G * R) return fail(ctx, BT_EINVAL, "bt_get_state: system out of range");
    g = system / R;
    r = system % R;
  } else {
    if (system < ctx->last_rb || system >= ctx->last_rb + ctx->last_Rs)
      return fail(ctx, BT_EINVAL, "bt_get_state: system not in the last run's RHS range");
    r = system - ctx->last_rb;
  }
  const int64_t row0 = ctx->seg_row0[g], rows = ctx->seg_row0[g + 1] - row0;
  if (n_rows) *n_rows = rows;
  if (!u_re_im) return BT_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  CK(ensure(ctx->d_state, (size_t)rows));
  const void* u = ctx->last_kind == 2 ? (const void*)ctx->udf.p : (const void*)ctx->u64.p;
  launch_extract_state(u, ctx->last_kind == 2, row0, rows, ctx->last_Rp, col_of_sys(r, ctx->last_nb),
                       ctx->d_state.p, ctx->sms, st);
  CKL();
  CK(cudaMemcpyAsync(u_re_im, ctx->d_state.p, (size_t)rows * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return BT_OK;
} BT_ABI_CATCH(ctx)

extern "C" bt_status bt_get_tuning(const bt_ctx* ctx, int32_t* variant, double* ms_iter, int32_t* resid_variant,
                                   double* ms_resid) {
  if (!ctx) return BT_EINVAL;
  if (ctx->tuned.empty()) return BT_ESTATE;
  const auto& t = ctx->tuned.back();
  if (variant) *variant = ctx->last_variant >= 0 ? ctx->last_variant : t.variant;
  if (resid_variant) *resid_variant = ctx->last_variant >= 0 ? ctx->last_resid_halo : (t.resid_halo ? 1 : 0);
  for (int k = 0; k < 2 + SLICE_NCONF; ++k)
    if (ms_iter) ms_iter[k] = t.ms[k];
  for (int k = 0; k < 2; ++k)
    if (ms_resid) ms_resid[k] = t.ms_resid[k];
  return BT_OK;
}

extern "C" bt_status bt_get_segment_stats(const bt_ctx* ctx, int32_t G, int64_t* sys_iters) {
  if (!ctx || !sys_iters || G < 1) return BT_EINVAL;
  if ((size_t)G != ctx->st_seg_sys_iters.size()) return BT_EINVAL;
  for (int32_t g = 0; g < G; ++g) sys_iters[g] = (int64_t)ctx->st_seg_sys_iters[g];
  return BT_OK;
}

extern "C" bt_status bt_get_stats(const bt_ctx* ctx, int64_t* steps, int64_t* krylov_iters, int64_t* refine_passes,
                                  int64_t* spmm_launches, double* spmm_ms, double* resid_ms,
                                  int64_t* resid_launches, int64_t* kernel_launches, int64_t* sys_iters,
                                  double* vec_ms) {
  if (!ctx) return BT_EINVAL;
  if (steps) *steps = ctx->st_steps;
  if (krylov_iters) *krylov_iters = ctx->st_iters;
  if (refine_passes) *refine_passes = ctx->st_refine;
  if (spmm_launches) *spmm_launches = ctx->st_spmm;
  if (spmm_ms) *spmm_ms = ctx->st_spmm_ms;
  if (resid_ms) *resid_ms = ctx->st_resid_ms;
  if (resid_launches) *resid_launches = ctx->st_resid;
  if (kernel_launches) *kernel_launches = ctx->st_launches;
  if (sys_iters) *sys_iters = ctx->st_sys_iters;
  if (vec_ms) *vec_ms = ctx->st_vec_ms;
  return BT_OK;
}
