// C ABI of the learned polynomial preconditioner: training on the GPU with
// the library's own forward/backward/Adam kernels, evaluation (coefficients,
// loss and gradient for given samples), weight save/load, and the geometry
// features of the current mesh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bt_ctx.h"

using namespace bt;

namespace {

struct XorShift {
  uint64_t s;
  explicit XorShift(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull) {
    if (!s) s = 1;
  }
  uint64_t next() {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    return s * 0x2545F4914F6CDD1Dull;
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

// c* = G^-1 h by Gaussian elimination with partial pivoting; false if singular
bool solve9(const double* G, const double* h, double* c) {
  double A[9][10];
  for (int i = 0; i < 9; ++i) {
    for (int j = 0; j < 9; ++j) A[i][j] = G[9 * i + j];
    A[i][9] = h[i];
  }
  for (int k = 0; k < 9; ++k) {
    int p = k;
    for (int i = k + 1; i < 9; ++i)
      if (std::fabs(A[i][k]) > std::fabs(A[p][k])) p = i;
    if (!(std::fabs(A[p][k]) > 1e-300)) return false;
    if (p != k)
      for (int j = 0; j < 10; ++j) std::swap(A[k][j], A[p][j]);
    for (int i = k + 1; i < 9; ++i) {
      const double f = A[i][k] / A[k][k];
      for (int j = k; j < 10; ++j) A[i][j] -= f * A[k][j];
    }
  }
  for (int i = 8; i >= 0; --i) {
    double s = A[i][9];
    for (int j = i + 1; j < 9; ++j) s -= A[i][j] * c[j];
    c[i] = s / A[i][i];
  }
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(c[i])) return false;
  return true;
}

bt_status ensure_precond_buffers(bt_ctx* ctx) {
  CK(ensure(ctx->pw32, MLP_NPARAM));
  CK(ensure(ctx->pw16, MLP_NPARAM));
  CK(ensure(ctx->pm, MLP_NPARAM));
  CK(ensure(ctx->pv, MLP_NPARAM));
  return BT_OK;
}

}  // namespace

namespace bt {
// volume-weighted mean D, area-weighted mean interface kappa (0 without
// interfaces), and h = (6 * mean tetrahedron volume)^(1/3)
void compute_geom_features(bt_ctx* ctx) {
  const HostMesh& m = ctx->mesh;
  double vol = 0, dv = 0;
  if (m.nv == 2) {
    // 1-D manifold: lengths, no membranes, h = mean segment length
    for (int64_t t = 0; t < m.n_tets; ++t) {
      const double* a = &m.xyz[3 * m.tets[2 * t]];
      const double* b = &m.xyz[3 * m.tets[2 * t + 1]];
      const double l =
          std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
      vol += l;
      dv += l * m.D[m.tet_cmpt[t]];
    }
    ctx->feat_D = vol > 0 ? dv / vol : 0;
    ctx->feat_kappa = 0;
    ctx->feat_h = vol / std::max<int64_t>(1, m.n_tets);
    return;
  }
  if (m.nv == 3) {
    // 2-D or surface: areas, interface edge lengths, h = (2 x mean triangle area)^(1/2)
    for (int64_t t = 0; t < m.n_tets; ++t) {
      const int32_t* v = &m.tets[3 * t];
      const double* a = &m.xyz[3 * v[0]];
      const double* b = &m.xyz[3 * v[1]];
      const double* c = &m.xyz[3 * v[2]];
      double A = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));
      if (m.surface) {
        const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2], n2 = u[0] * w[1] - u[1] * w[0];
        A = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
      }
      vol += A;
      dv += A * m.D[m.tet_cmpt[t]];
    }
    double len = 0, kl = 0;
    for (int64_t f = 0; f < m.n_face; ++f) {
      const int32_t t = m.face_ta[f];
      const double* a = &m.xyz[3 * m.tets[3 * t + m.face_lv[2 * f]]];
      const double* b = &m.xyz[3 * m.tets[3 * t + m.face_lv[2 * f + 1]]];
      const double l =
          std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
      len += l;
      kl += l * m.face_kappa[f];
    }
    ctx->feat_D = vol > 0 ? dv / vol : 0;
    ctx->feat_kappa = len > 0 ? kl / len : 0;
    ctx->feat_h = std::sqrt(2.0 * vol / std::max<int64_t>(1, m.n_tets));
    return;
  }
  for (int64_t t = 0; t < m.n_tets; ++t) {
    const int32_t* v = &m.tets[4 * t];
    const double* a = &m.xyz[3 * v[0]];
    const double* b = &m.xyz[3 * v[1]];
    const double* c = &m.xyz[3 * v[2]];
    const double* d = &m.xyz[3 * v[3]];
    double e1[3], e2[3], e3[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = b[k] - a[k];
      e2[k] = c[k] - a[k];
      e3[k] = d[k] - a[k];
    }
    const double V = ((e1[1] * e2[2] - e1[2] * e2[1]) * e3[0] + (e1[2] * e2[0] - e1[0] * e2[2]) * e3[1] +
                      (e1[0] * e2[1] - e1[1] * e2[0]) * e3[2]) / 6.0;
    vol += V;
    dv += V * m.D[m.tet_cmpt[t]];
  }
  double area = 0, ka = 0;
  for (int64_t f = 0; f < m.n_face; ++f) {
    const int32_t t = m.face_ta[f];
    double P[3][3];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) P[a][k] = m.xyz[3 * m.tets[4 * t + m.face_lv[3 * f + a]] + k];
    double u[3], w[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = P[1][k] - P[0][k];
      w[k] = P[2][k] - P[0][k];
    }
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
    const double A = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    area += A;
    ka += A * m.face_kappa[f];
  }
  ctx->feat_D = vol > 0 ? dv / vol : 0;
  ctx->feat_kappa = area > 0 ? ka / area : 0;
  ctx->feat_h = std::cbrt(6.0 * vol / std::max<int64_t>(1, m.n_tets));
}
}  // namespace bt

extern "C" {

bt_status bt_precond_features(const bt_ctx* ctx, double* D, double* kappa, double* h) {
  if (!ctx || !ctx->assembled) return BT_ESTATE;
  if (D) *D = ctx->feat_D;
  if (kappa) *kappa = ctx->feat_kappa;
  if (h) *h = ctx->feat_h;
  return BT_OK;
}

bt_status bt_train_default_opts(bt_train_opts* o) {
  if (!o) return BT_EINVAL;
  o->epochs = 300;
  o->batch = 512;
  o->lr = 2e-3;
  o->seed = 1;
  o->flags = 0;
  o->rel_err = 1e-6;
  return BT_OK;
}

bt_status bt_save_precond(const bt_ctx* ctx_c, float* w) {
  bt_ctx* ctx = const_cast<bt_ctx*>(ctx_c);
  if (!ctx || !w) return BT_EINVAL;
  if (!ctx->have_precond) return fail(ctx, BT_ESTATE, "bt_save_precond: no trained preconditioner");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(w, ctx->pw32.p, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return BT_OK;
}

bt_status bt_load_precond(bt_ctx* ctx, const float* w) try {
  if (!ctx || !w) return BT_EINVAL;
  if (ctx->host_only) return fail(ctx, BT_ENODEV, "bt_load_precond: host-only context");
  for (int i = 0; i < MLP_NPARAM; ++i)
    if (!std::isfinite(w[i])) return fail(ctx, BT_EINVAL, "bt_load_precond: non-finite weight");
  CK(cudaSetDevice(ctx->device));
  if (bt_status e = ensure_precond_buffers(ctx)) return e;
  CK(cudaMemcpyAsync(ctx->pw32.p, w, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  launch_to_bf16(ctx->pw32.p, ctx->pw16.p, MLP_NPARAM, ctx->stream);
  CKL();
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_precond = true;
  return BT_OK;
} BT_ABI_CATCH(ctx)

bt_status bt_set_precond_poly(bt_ctx* ctx, const double* c9) {
  if (!ctx) return BT_EINVAL;
  if (!c9) {
    ctx->have_fixed_poly = false;
    return BT_OK;
  }
  for (int j = 0; j < 9; ++j)
    if (!std::isfinite(c9[j])) return fail(ctx, BT_EINVAL, "bt_set_precond_poly: non-finite coefficient");
  std::copy(c9, c9 + 9, ctx->fixed_poly);
  ctx->have_fixed_poly = true;
  return BT_OK;
}

bt_status bt_get_precond_stats(const bt_ctx* ctx, int64_t* horner_launches) {
  if (!ctx) return BT_EINVAL;
  if (horner_launches) *horner_launches = ctx->st_horner;
  return BT_OK;
}

// Train the network on n samples (raw features [n][5], G [n][81], h [n][9])
// with minibatch Adam; loss_hist[epoch] receives the mean training loss.
bt_status bt_train_precond(bt_ctx* ctx, int64_t n, const float* feat, const double* G, const double* h,
                           const bt_train_opts* opts, double* loss_hist) try {
  if (!ctx) return BT_EINVAL;
  if (ctx->host_only) return fail(ctx, BT_ENODEV, "bt_train_precond: host-only context");
  bt_train_opts o;
  bt_train_default_opts(&o);
  if (opts) o = *opts;
  if (n < 1 || !feat || !G || !h || o.epochs < 1 || o.batch < 1 || !(o.lr > 0) || !(o.rel_err >= 0) ||
      !(o.rel_err < 1))
    return fail(ctx, BT_EINVAL, "bt_train_precond: bad arguments");
  const int B = (int)std::min<int64_t>(o.batch, n);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  if (bt_status e = ensure_precond_buffers(ctx)) return e;
  std::vector<float> Gf(81 * n), hf(9 * n);
  for (int64_t i = 0; i < 81 * n; ++i) Gf[i] = (float)G[i];
  for (int64_t i = 0; i < 9 * n; ++i) hf[i] = (float)h[i];
  DBuf<float> dfe, dG, dh, sx, sa1, sa2, sd1, sd2, sdc, dloss;
  DBuf<int> didx;
  CK(dfe.alloc(5 * n));
  CK(dG.alloc(81 * n));
  CK(dh.alloc(9 * n));
  CK(didx.alloc(n));
  const int64_t steps_per_epoch = n / B;
  CK(dloss.alloc(steps_per_epoch * B));
  CK(sx.alloc((size_t)B * MLP_IN));
  CK(sa1.alloc((size_t)B * MLP_H));
  CK(sa2.alloc((size_t)B * MLP_H));
  CK(sd1.alloc((size_t)B * MLP_H));
  CK(sd2.alloc((size_t)B * MLP_H));
  CK(sdc.alloc((size_t)B * MLP_OUT));
  CK(cudaMemcpyAsync(dfe.p, feat, 5 * n * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dG.p, Gf.data(), 81 * n * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dh.p, hf.data(), 9 * n * sizeof(float), cudaMemcpyHostToDevice, st));

  XorShift rng(o.seed);
  if (!(o.flags & BT_TRAIN_CONTINUE) || !ctx->have_precond) {
    // He-uniform hidden layers, small output layer, output bias = mean of the
    // per-sample optimal coefficients (a good starting polynomial)
    std::vector<float> w(MLP_NPARAM, 0.f);
    const int OW1 = 0, OB1 = OW1 + MLP_H * MLP_IN, OW2 = OB1 + MLP_H, OB2 = OW2 + MLP_H * MLP_H,
              OW3 = OB2 + MLP_H, OB3 = OW3 + MLP_OUT * MLP_H;
    (void)OB2;
    const double a1 = std::sqrt(6.0 / MLP_IN), a2 = std::sqrt(6.0 / MLP_H);
    for (int i = OW1; i < OB1; ++i) w[i] = (float)((2 * rng.uniform() - 1) * a1);
    for (int i = OW2; i < OW2 + MLP_H * MLP_H; ++i) w[i] = (float)((2 * rng.uniform() - 1) * a2);
    for (int i = OW3; i < OB3; ++i) w[i] = (float)((2 * rng.uniform() - 1) * 0.01);
    double cm[9] = {0}, c[9];
    int64_t good = 0;
    for (int64_t s = 0; s < n; ++s)
      if (solve9(G + 81 * s, h + 9 * s, c)) {
        for (int j = 0; j < 9; ++j) cm[j] += c[j];
        ++good;
      }
    for (int j = 0; j < 9; ++j) w[OB3 + j] = good ? (float)(cm[j] / good) : (j == 0 ? 1.f : 0.f);
    CK(cudaMemcpyAsync(ctx->pw32.p, w.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    launch_to_bf16(ctx->pw32.p, ctx->pw16.p, MLP_NPARAM, st);
    CKL();
    CK(cudaMemsetAsync(ctx->pm.p, 0, MLP_NPARAM * sizeof(float), st));
    CK(cudaMemsetAsync(ctx->pv.p, 0, MLP_NPARAM * sizeof(float), st));
  }
  std::vector<int> perm(n);
  std::vector<float> lh(steps_per_epoch * B);
  int t = 0;
  for (int ep = 0; ep < o.epochs; ++ep) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
    for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)(rng.uniform() * (i + 1)) % (i + 1)]);
    CK(cudaMemcpyAsync(didx.p, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    for (int64_t k = 0; k < steps_per_epoch; ++k) {
      MlpTrainArgs a{};
      a.w32 = ctx->pw32.p;
      a.w16 = ctx->pw16.p;
      a.m = ctx->pm.p;
      a.v = ctx->pv.p;
      a.feat = dfe.p;
      a.G = dG.p;
      a.h = dh.p;
      a.idx = didx.p + k * B;
      a.B = B;
      a.sx = sx.p;
      a.sa1 = sa1.p;
      a.sa2 = sa2.p;
      a.sd1 = sd1.p;
      a.sd2 = sd2.p;
      a.sdc = sdc.p;
      a.loss = dloss.p + k * B;
      a.grad_out = nullptr;
      a.apply = 1;
      a.t = ++t;
      a.lr = (float)o.lr;
      a.beta1 = 0.9f;
      a.beta2 = 0.999f;
      a.eps = 1e-8f;
      a.rel_err = (float)o.rel_err;
      launch_mlp_train(a, st);
      CKL();
    }
    CK(cudaMemcpyAsync(lh.data(), dloss.p, lh.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double sum = 0;
    for (float v : lh) sum += v;
    if (loss_hist) loss_hist[ep] = sum / std::max<size_t>(1, lh.size());
  }
  CK(cudaStreamSynchronize(st));
  ctx->have_precond = true;
  return BT_OK;
} BT_ABI_CATCH(ctx)

// For n samples: coefficients [n][9] from the current network, the mean loss
// and its gradient with respect to the parameters [MLP_NPARAM] (through the
// bfloat16 weights).  Any output pointer may be NULL.
bt_status bt_precond_eval(bt_ctx* ctx, int64_t n, const float* feat, const double* G, const double* h,
                          double rel_err, double* coef, double* loss, double* grad) try {
  if (!ctx || n < 1 || !feat || !(rel_err >= 0) || !(rel_err < 1))
    return fail(ctx, BT_EINVAL, "bt_precond_eval: bad arguments");
  if (ctx->host_only) return fail(ctx, BT_ENODEV, "bt_precond_eval: host-only context");
  if (!ctx->have_precond) return fail(ctx, BT_ESTATE, "bt_precond_eval: no network");
  if ((loss || grad) && (!G || !h)) return fail(ctx, BT_EINVAL, "bt_precond_eval: loss needs G and h");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DBuf<float> dfe;
  CK(dfe.alloc(5 * n));
  CK(cudaMemcpyAsync(dfe.p, feat, 5 * n * sizeof(float), cudaMemcpyHostToDevice, st));
  if (coef) {
    DBuf<double> dc;
    CK(dc.alloc(9 * n));
    launch_mlp_forward(ctx->pw16.p, dfe.p, (int)n, dc.p, st);
    CKL();
    CK(cudaMemcpyAsync(coef, dc.p, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (loss || grad) {
    std::vector<float> Gf(81 * n), hf(9 * n);
    for (int64_t i = 0; i < 81 * n; ++i) Gf[i] = (float)G[i];
    for (int64_t i = 0; i < 9 * n; ++i) hf[i] = (float)h[i];
    std::vector<int> idx(n);
    for (int64_t i = 0; i < n; ++i) idx[i] = (int)i;
    DBuf<float> dG, dh, sx, sa1, sa2, sd1, sd2, sdc, dl;
    DBuf<int> di;
    DBuf<double> dg;
    CK(dG.alloc(81 * n));
    CK(dh.alloc(9 * n));
    CK(di.alloc(n));
    CK(sx.alloc(n * MLP_IN));
    CK(sa1.alloc(n * MLP_H));
    CK(sa2.alloc(n * MLP_H));
    CK(sd1.alloc(n * MLP_H));
    CK(sd2.alloc(n * MLP_H));
    CK(sdc.alloc(n * MLP_OUT));
    CK(dl.alloc(n));
    CK(dg.alloc(MLP_NPARAM));
    CK(cudaMemcpyAsync(dG.p, Gf.data(), 81 * n * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dh.p, hf.data(), 9 * n * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(di.p, idx.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    MlpTrainArgs a{};
    a.w32 = ctx->pw32.p;
    a.w16 = ctx->pw16.p;
    a.m = ctx->pm.p;
    a.v = ctx->pv.p;
    a.feat = dfe.p;
    a.G = dG.p;
    a.h = dh.p;
    a.idx = di.p;
    a.B = (int)n;
    a.sx = sx.p;
    a.sa1 = sa1.p;
    a.sa2 = sa2.p;
    a.sd1 = sd1.p;
    a.sd2 = sd2.p;
    a.sdc = sdc.p;
    a.loss = dl.p;
    a.grad_out = dg.p;
    a.apply = 0;
    a.rel_err = (float)rel_err;
    launch_mlp_train(a, st);
    CKL();
    std::vector<float> lv(n);
    CK(cudaMemcpyAsync(lv.data(), dl.p, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (grad) CK(cudaMemcpyAsync(grad, dg.p, MLP_NPARAM * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (loss) {
      double s = 0;
      for (float v : lv) s += v;
      *loss = s / n;
    }
  }
  return BT_OK;
} BT_ABI_CATCH(ctx)

}  // extern "C"
