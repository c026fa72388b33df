// Deterministic element-by-element assembly of every matrix of the method over
// one shared CSR pattern (no floating-point atomics: each slot sums its
// element contributions in a fixed, increasing element order).
//
// Element matrices of P1 tetrahedra with volume |T| and barycentric gradients
// G (rows grad lambda_i), exact integration:
//   M_ij  = |T|/20 (1 + delta_ij)                       mass       (Appendix B, M)
//   K_ij  = D |T| G_i . G_j                             stiffness  (Appendix B, S)
//   Mk_ij = |T| sum_l x_{l,k} int(lambda_i lambda_j lambda_l)/|T|  first moment
//           (Appendix B, J = (g.x U, v)); the cubic integrals are
//           1/20 (i=j=l), 1/60 (two equal), 1/120 (all distinct), which gives
//           (2 x_i + S)/60 for i = j and (S + x_i + x_j)/120 otherwise, S = sum_l x_l
//   Ek_ij = C_k,ij - C_k,ji, C_k,ij = D |T|/4 G_j,k     transformed frame (Appendix A)
// Interface faces (area |F|, permeability kappa):
//   J += kappa |F|/12 (1 + delta) [[+1, -1], [-1, +1]] over (side a, side b) dofs
//   (Appendix B, I = kappa <[U], [v]>).
#include "bt_kernels.cuh"

namespace bt {

// geometry record of one tetrahedron: vol, G[4][3], Xc[4][3] (relative to the
// box centre), D, 1/T2, diffusion tensor (xx, yy, zz, xy, yz, zx): the
// element's own (DtenE, cell-based), else its compartment's (Dten), else D I
static constexpr int TG = 33;

__global__ void k_tet_geom(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                           const int32_t* __restrict__ cmpt, const double* __restrict__ Dc,
                           const double* __restrict__ invT2c, const double* __restrict__ Dten, double cx,
                           double cy, double cz, int64_t nt, double* __restrict__ out,
                           const double* __restrict__ DtenE) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[4][3];
  for (int a = 0; a < 4; ++a) {
    int64_t v = tets[4 * t + a];
    X[a][0] = xyz[3 * v + 0];
    X[a][1] = xyz[3 * v + 1];
    X[a][2] = xyz[3 * v + 2];
  }
  double E[3][3];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) E[a][k] = X[a + 1][k] - X[0][k];
  // cofactors: inverse of E has columns grad lambda_{1..3}
  double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
  double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
  double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
  double det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
  double id = 1.0 / det;
  // grad lambda_{a+1} = (row a of cofactor-of-E^T) / det: components of the
  // dual basis g_a with g_a . e_b = delta_ab, e_b = row b of E
  double g[3][3];
  // g_0 = (e1 x e2)/det, g_1 = (e2 x e0)/det, g_2 = (e0 x e1)/det
  const double* e0 = E[0];
  const double* e1 = E[1];
  const double* e2 = E[2];
  g[0][0] = (e1[1] * e2[2] - e1[2] * e2[1]) * id;
  g[0][1] = (e1[2] * e2[0] - e1[0] * e2[2]) * id;
  g[0][2] = (e1[0] * e2[1] - e1[1] * e2[0]) * id;
  g[1][0] = (e2[1] * e0[2] - e2[2] * e0[1]) * id;
  g[1][1] = (e2[2] * e0[0] - e2[0] * e0[2]) * id;
  g[1][2] = (e2[0] * e0[1] - e2[1] * e0[0]) * id;
  g[2][0] = (e0[1] * e1[2] - e0[2] * e1[1]) * id;
  g[2][1] = (e0[2] * e1[0] - e0[0] * e1[2]) * id;
  g[2][2] = (e0[0] * e1[1] - e0[1] * e1[0]) * id;
  (void)c00; (void)c01; (void)c02;
  double* o = out + TG * t;
  o[0] = det / 6.0;
  for (int k = 0; k < 3; ++k) {
    o[1 + k] = -(g[0][k] + g[1][k] + g[2][k]);
    o[4 + k] = g[0][k];
    o[7 + k] = g[1][k];
    o[10 + k] = g[2][k];
  }
  const double c[3] = {cx, cy, cz};
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) o[13 + 3 * a + k] = X[a][k] - c[k];
  const int cm = cmpt[t];
  o[25] = Dc[cm];
  o[26] = invT2c ? invT2c[cm] : 0.0;
  for (int k = 0; k < 6; ++k)
    o[27 + k] = DtenE ? DtenE[6 * t + k] : Dten ? Dten[6 * cm + k] : (k < 3 ? Dc[cm] : 0.0);
}

// The same record for a triangle in the xy plane (2-D meshes): area, the
// gradients of the three barycentric coordinates (z = 0), the vertices
// relative to the box centre; the fourth vertex slots are zero.
__global__ void k_tri_geom(const double* __restrict__ xyz, const int32_t* __restrict__ tris,
                           const int32_t* __restrict__ cmpt, const double* __restrict__ Dc,
                           const double* __restrict__ invT2c, const double* __restrict__ Dten, double cx,
                           double cy, double cz, int64_t nt, double* __restrict__ out,
                           const double* __restrict__ DtenE) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[3][3];
  for (int a = 0; a < 3; ++a) {
    int64_t v = tris[3 * t + a];
    for (int k = 0; k < 3; ++k) X[a][k] = xyz[3 * v + k];
  }
  const double area2 = (X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) - (X[1][1] - X[0][1]) * (X[2][0] - X[0][0]);
  const double id = 1.0 / area2;
  double* o = out + TG * t;
  for (int k = 0; k < TG; ++k) o[k] = 0.0;
  o[0] = 0.5 * area2;
  // grad lambda_a = perp(x_{a+2} - x_{a+1}) / (2 area), indices mod 3
  for (int a = 0; a < 3; ++a) {
    const double* p = X[(a + 1) % 3];
    const double* q = X[(a + 2) % 3];
    o[1 + 3 * a + 0] = (p[1] - q[1]) * id;
    o[1 + 3 * a + 1] = (q[0] - p[0]) * id;
  }
  const double c[3] = {cx, cy, cz};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) o[13 + 3 * a + k] = X[a][k] - c[k];
  const int cm = cmpt[t];
  o[25] = Dc[cm];
  o[26] = invT2c ? invT2c[cm] : 0.0;
  for (int k = 0; k < 6; ++k)
    o[27 + k] = DtenE ? DtenE[6 * t + k] : Dten ? Dten[6 * cm + k] : (k < 3 ? Dc[cm] : 0.0);
}

// The record for a triangle of a surface embedded in 3-D (a thin layer): area,
// the tangential gradients grad lambda_a = n x (x_{a+2} - x_{a+1}) / |n|^2 with
// n = (x_1 - x_0) x (x_2 - x_0) (indices mod 3; for a counter-clockwise
// triangle of the xy plane this is the planar formula), the vertices relative
// to the box centre; the fourth vertex slots are zero.
__global__ void k_stri_geom(const double* __restrict__ xyz, const int32_t* __restrict__ tris,
                            const int32_t* __restrict__ cmpt, const double* __restrict__ Dc,
                            const double* __restrict__ invT2c, const double* __restrict__ Dten, double cx,
                            double cy, double cz, int64_t nt, double* __restrict__ out,
                           const double* __restrict__ DtenE) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[3][3];
  for (int a = 0; a < 3; ++a) {
    int64_t v = tris[3 * t + a];
    for (int k = 0; k < 3; ++k) X[a][k] = xyz[3 * v + k];
  }
  double u[3], w[3];
  for (int k = 0; k < 3; ++k) {
    u[k] = X[1][k] - X[0][k];
    w[k] = X[2][k] - X[0][k];
  }
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  double* o = out + TG * t;
  for (int k = 0; k < TG; ++k) o[k] = 0.0;
  o[0] = 0.5 * sqrt(n2);
  for (int a = 0; a < 3; ++a) {
    const double* p = X[(a + 1) % 3];
    const double* q = X[(a + 2) % 3];
    const double e[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    o[1 + 3 * a + 0] = (n[1] * e[2] - n[2] * e[1]) / n2;
    o[1 + 3 * a + 1] = (n[2] * e[0] - n[0] * e[2]) / n2;
    o[1 + 3 * a + 2] = (n[0] * e[1] - n[1] * e[0]) / n2;
  }
  const double c[3] = {cx, cy, cz};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) o[13 + 3 * a + k] = X[a][k] - c[k];
  const int cm = cmpt[t];
  o[25] = Dc[cm];
  o[26] = invT2c ? invT2c[cm] : 0.0;
  for (int k = 0; k < 6; ++k)
    o[27 + k] = DtenE ? DtenE[6 * t + k] : Dten ? Dten[6 * cm + k] : (k < 3 ? Dc[cm] : 0.0);
}

// The record for a segment of a 1-D manifold embedded in 3-D: length, the
// tangential gradients -+ e / |e|^2 of the two barycentric coordinates, the
// vertices relative to the box centre; the other vertex slots are zero.
__global__ void k_seg_geom(const double* __restrict__ xyz, const int32_t* __restrict__ segs,
                           const int32_t* __restrict__ cmpt, const double* __restrict__ Dc,
                           const double* __restrict__ invT2c, const double* __restrict__ Dten, double cx,
                           double cy, double cz, int64_t nt, double* __restrict__ out,
                           const double* __restrict__ DtenE) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[2][3];
  for (int a = 0; a < 2; ++a) {
    int64_t v = segs[2 * t + a];
    for (int k = 0; k < 3; ++k) X[a][k] = xyz[3 * v + k];
  }
  double e[3], l2 = 0;
  for (int k = 0; k < 3; ++k) {
    e[k] = X[1][k] - X[0][k];
    l2 += e[k] * e[k];
  }
  double* o = out + TG * t;
  for (int k = 0; k < TG; ++k) o[k] = 0.0;
  o[0] = sqrt(l2);
  for (int k = 0; k < 3; ++k) {
    o[1 + k] = -e[k] / l2;
    o[4 + k] = e[k] / l2;
  }
  const double c[3] = {cx, cy, cz};
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) o[13 + 3 * a + k] = X[a][k] - c[k];
  const int cm = cmpt[t];
  o[25] = Dc[cm];
  o[26] = invT2c ? invT2c[cm] : 0.0;
  for (int k = 0; k < 6; ++k)
    o[27 + k] = DtenE ? DtenE[6 * t + k] : Dten ? Dten[6 * cm + k] : (k < 3 ? Dc[cm] : 0.0);
}

// kappa |F| / 12 per interface face (3-D); kappa |e| / 6 per interface edge (2-D)
__global__ void k_face_coef(const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                            const int32_t* __restrict__ ta, const int8_t* __restrict__ lv,
                            const double* __restrict__ kap, int64_t nf, int nv, double* __restrict__ out) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  if (nv == 3) {
    const int64_t v0 = tets[3 * (int64_t)ta[f] + lv[2 * f]], v1 = tets[3 * (int64_t)ta[f] + lv[2 * f + 1]];
    double l2 = 0;
    for (int k = 0; k < 3; ++k) l2 += (xyz[3 * v1 + k] - xyz[3 * v0 + k]) * (xyz[3 * v1 + k] - xyz[3 * v0 + k]);
    out[f] = kap[f] * sqrt(l2) / 6.0;
    return;
  }
  double P[3][3];
  for (int a = 0; a < 3; ++a) {
    int64_t v = tets[4 * (int64_t)ta[f] + lv[3 * f + a]];
    for (int k = 0; k < 3; ++k) P[a][k] = xyz[3 * v + k];
  }
  double u[3], w[3];
  for (int k = 0; k < 3; ++k) {
    u[k] = P[1][k] - P[0][k];
    w[k] = P[2][k] - P[0][k];
  }
  double cx = u[1] * w[2] - u[2] * w[1];
  double cy = u[2] * w[0] - u[0] * w[2];
  double cz = u[0] * w[1] - u[1] * w[0];
  double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  out[f] = kap[f] * area / 12.0;
}

// One thread per slot of the pattern: sums that slot's tetrahedron and face
// contributions (in increasing element order) into the eleven value planes
// M, K, J, MD, Mx, My, Mz, Ex, Ey, Ez, MR (plane stride nnz); MR is the mass
// weighted by 1/T2 of each element's compartment (the relaxation term
// (U / T2, v) of the weak form).
__global__ void k_assemble_slots(const double* __restrict__ geo, const int64_t* __restrict__ tc_ptr,
                                 const int32_t* __restrict__ tc, const int64_t* __restrict__ fc_ptr,
                                 const int32_t* __restrict__ fc, const double* __restrict__ fcoef,
                                 int64_t nnz, int nv, double* __restrict__ planes) {
  // element integrals over a d-simplex (exact for P1):
  //   int l_i l_j = |T| (1 + d_ij) / ((d+1)(d+2)),   int l_i = |T| / (d + 1),
  //   int l_i l_j l_l = |T| d! a! b! c! / (d + a + b + c)!, which makes
  //   int l_i^2 x = 2 |T| (S + 2 x_i) d! / (d+3)!,  int l_i l_j x = |T| (S + x_i + x_j) d! / (d+3)!
  //   with S the sum of the element's vertices (unused vertex slots hold zero)
  const int d = nv - 1;
  const double m_off = 1.0 / ((d + 1) * (d + 2)), m_diag = 2.0 * m_off;
  const double mom_o = d == 3 ? 120.0 : d == 2 ? 60.0 : 24.0, mom_d = 0.5 * mom_o, c_int = 1.0 / (d + 1);
  const int n2 = nv * nv, fs = nv - 1, nfd = 2 * fs;
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nnz) return;
  double m = 0, kk = 0, md = 0, mx = 0, my = 0, mz = 0, ex = 0, ey = 0, ez = 0, jj = 0, mr = 0;
  for (int64_t q = tc_ptr[s]; q < tc_ptr[s + 1]; ++q) {
    int32_t code = tc[q];
    int32_t t = code / n2;
    const int rr = code - n2 * t;
    int i = rr / nv, j = rr - nv * (rr / nv);
    const double* g = geo + (int64_t)TG * t;
    double vol = g[0], D = g[25], rT2 = g[26];
    const double* Gi = g + 1 + 3 * i;
    const double* Gj = g + 1 + 3 * j;
    const double* Xc = g + 13;
    double mass = vol * (i == j ? m_diag : m_off);
    m += mass;
    md += D * mass;
    mr += rT2 * mass;
    // (D grad phi_j) . grad phi_i with the element's symmetric tensor
    const double* T = g + 27;
    const double DG0 = T[0] * Gj[0] + T[3] * Gj[1] + T[5] * Gj[2];
    const double DG1 = T[3] * Gj[0] + T[1] * Gj[1] + T[4] * Gj[2];
    const double DG2 = T[5] * Gj[0] + T[4] * Gj[1] + T[2] * Gj[2];
    kk += vol * (Gi[0] * DG0 + Gi[1] * DG1 + Gi[2] * DG2);
    double mom[3];
    for (int k = 0; k < 3; ++k) {
      double S = Xc[k] + Xc[3 + k] + Xc[6 + k] + Xc[9 + k];
      mom[k] = (i == j) ? vol * (2.0 * Xc[3 * i + k] + S) / mom_d
                        : vol * (S + Xc[3 * i + k] + Xc[3 * j + k]) / mom_o;
    }
    mx += mom[0];
    my += mom[1];
    mz += mom[2];
    double c4 = D * vol * c_int;
    ex += c4 * (Gj[0] - Gi[0]);
    ey += c4 * (Gj[1] - Gi[1]);
    ez += c4 * (Gj[2] - Gi[2]);
  }
  for (int64_t q = fc_ptr[s]; q < fc_ptr[s + 1]; ++q) {
    int32_t code = fc[q];
    int32_t f = code / (nfd * nfd);
    int r = code - nfd * nfd * f;
    int a = r / nfd, b = r - nfd * a;
    double v = fcoef[f] * ((a % fs) == (b % fs) ? 2.0 : 1.0);
    jj += ((a < fs) == (b < fs)) ? v : -v;
  }
  planes[0 * nnz + s] = m;
  planes[1 * nnz + s] = kk;
  planes[2 * nnz + s] = jj;
  planes[3 * nnz + s] = md;
  planes[4 * nnz + s] = mx;
  planes[5 * nnz + s] = my;
  planes[6 * nnz + s] = mz;
  planes[7 * nnz + s] = ex;
  planes[8 * nnz + s] = ey;
  planes[9 * nnz + s] = ez;
  planes[10 * nnz + s] = mr;
}

// Step planes for theta and dt, per slot:
//   A0 = M + theta dt (K + J + MR + MB), KJ = K + J + MR + theta MB
//   (MR = 0 without relaxation, MB = 0 without the weak periodic box)
//   pk64 = {A0, d0, d1, d2} (FP64), pk32 = same in FP32,
//   direction planes d = (Mx,My,Mz) in the lab frame, (Ex,Ey,Ez) transformed.
__global__ void k_derive_planes(const double* __restrict__ planes, const double* __restrict__ MB, double theta,
                                int64_t nnz, double thdt, int transformed,
                                double* __restrict__ A0, double* __restrict__ KJ, double4* __restrict__ pk64,
                                float4* __restrict__ pk32, float* __restrict__ md32,
                                float4* __restrict__ pkhi, float4* __restrict__ pklo,
                                float2* __restrict__ kjmd_hi, float2* __restrict__ kjmd_lo) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nnz) return;
  double m = planes[s], k = planes[nnz + s], j = planes[2 * nnz + s], md = planes[3 * nnz + s];
  int o = transformed ? 7 : 4;
  double d0 = planes[(o + 0) * nnz + s], d1 = planes[(o + 1) * nnz + s], d2 = planes[(o + 2) * nnz + s];
  // the artificial-permeability boundary mass enters L with theta dt and the
  // step-start operator (R - L) with theta dt, i.e. P0 = K + J + MR + theta MB
  const double base = k + j + planes[10 * nnz + s];
  const double mb = MB ? MB[s] : 0.0;
  double kj = base + theta * mb;
  double a0 = m + thdt * (base + mb);
  A0[s] = a0;
  KJ[s] = kj;
  pk64[s] = make_double4(a0, d0, d1, d2);
  pk32[s] = make_float4((float)a0, (float)d0, (float)d1, (float)d2);
  md32[s] = (float)md;
  float h0 = (float)a0, h1 = (float)d0, h2 = (float)d1, h3 = (float)d2;
  pkhi[s] = make_float4(h0, h1, h2, h3);
  pklo[s] = make_float4((float)(a0 - h0), (float)(d0 - h1), (float)(d1 - h2), (float)(d2 - h3));
  float hk = (float)kj, hm = (float)md;
  kjmd_hi[s] = make_float2(hk, hm);
  kjmd_lo[s] = make_float2((float)(kj - hk), (float)(md - hm));
}

// Per row: signal weight w_i = sum_j M_ij (Eq. signal: exact integral of the
// basis function) and the diagonal entries used by the Jacobi preconditioner.
__global__ void k_row_data(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ planes, const double4* __restrict__ pk64,
                           int64_t nnz, int64_t n, double* __restrict__ w, double4* __restrict__ diag64,
                           double* __restrict__ diag_md64, float4* __restrict__ diag32,
                           float* __restrict__ diag_md32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0;
  double4 dg = make_double4(0, 0, 0, 0);
  double dmd = 0;
  for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
    s += planes[q];
    if (col[q] == i) {
      dg = pk64[q];
      dmd = planes[3 * nnz + q];
    }
  }
  w[i] = s;
  diag64[i] = dg;
  diag_md64[i] = dmd;
  diag32[i] = make_float4((float)dg.x, (float)dg.y, (float)dg.z, (float)dg.w);
  diag_md32[i] = (float)dmd;
}

void launch_assembly(const AsmArgs& a, cudaStream_t st) {
  const int TB = 256;
  if (a.nt && a.nv == 4)
    k_tet_geom<<<(unsigned)((a.nt + TB - 1) / TB), TB, 0, st>>>(a.xyz, a.tets, a.cmpt, a.Dc, a.invT2c, a.Dten,
                                                              a.centre[0], a.centre[1], a.centre[2], a.nt, a.geo,
                                                              a.DtenE);
  if (a.nt && a.nv == 2)
    k_seg_geom<<<(unsigned)((a.nt + TB - 1) / TB), TB, 0, st>>>(a.xyz, a.tets, a.cmpt, a.Dc, a.invT2c, a.Dten,
                                                               a.centre[0], a.centre[1], a.centre[2], a.nt, a.geo,
                                                              a.DtenE);
  if (a.nt && a.nv == 3 && a.surface)
    k_stri_geom<<<(unsigned)((a.nt + TB - 1) / TB), TB, 0, st>>>(a.xyz, a.tets, a.cmpt, a.Dc, a.invT2c, a.Dten,
                                                               a.centre[0], a.centre[1], a.centre[2], a.nt, a.geo,
                                                              a.DtenE);
  if (a.nt && a.nv == 3 && !a.surface)
    k_tri_geom<<<(unsigned)((a.nt + TB - 1) / TB), TB, 0, st>>>(a.xyz, a.tets, a.cmpt, a.Dc, a.invT2c, a.Dten,
                                                              a.centre[0], a.centre[1], a.centre[2], a.nt, a.geo,
                                                              a.DtenE);
  if (a.nf) k_face_coef<<<(unsigned)((a.nf + TB - 1) / TB), TB, 0, st>>>(a.xyz, a.tets, a.face_ta, a.face_lv,
                                                                   a.face_kappa, a.nf, a.nv, a.fcoef);
  k_assemble_slots<<<(unsigned)((a.nnz + TB - 1) / TB), TB, 0, st>>>(a.geo, a.tc_ptr, a.tc, a.fc_ptr, a.fc,
                                                                    a.fcoef, a.nnz, a.nv, a.planes);
}

void launch_derive(const DeriveArgs& a, cudaStream_t st) {
  const int TB = 256;
  k_derive_planes<<<(unsigned)((a.nnz + TB - 1) / TB), TB, 0, st>>>(
      a.planes, a.MB, a.theta, a.nnz, a.thdt, a.transformed, a.A0, a.KJ, a.pk64, a.pk32, a.md32, a.pkhi, a.pklo, a.kjmd_hi,
      a.kjmd_lo);
  k_row_data<<<(unsigned)((a.n + TB - 1) / TB), TB, 0, st>>>(a.rp, a.col, a.planes, a.pk64, a.nnz, a.n, a.w,
                                                            a.diag64, a.diag_md64, a.diag32, a.diag_md32);
}

}  // namespace bt
