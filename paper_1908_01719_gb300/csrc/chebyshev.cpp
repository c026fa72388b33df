// Fixed Chebyshev polynomial preconditioner: the baseline a learned
// polynomial has to beat.  P = p(B) D^-1 with B = D^-1 L leaves the residual
// polynomial 1 - l p(l) on the spectrum of B; the degree-9 residual
// polynomial of least maximum modulus on [lo, hi] with value 1 at l = 0 is
//   r(l) = T_9((hi + lo - 2 l)/(hi - lo)) / T_9((hi + lo)/(hi - lo)),
// T_9 the Chebyshev polynomial of the first kind (T_0 = 1, T_1 = x,
// T_{k+1} = 2 x T_k - T_{k-1}), so p(l) = (1 - r(l))/l has degree 8 and its
// monomial coefficients c_0..c_8 are minus the coefficients r_1..r_9 of r.
// The interval is fitted to the step solves' own residual data: the
// per-sample loss |r - L P r|^2/|r|^2 = 1 - 2 c.h + c.G c (the quantity the
// network is trained on) averaged over the samples, minimised over (lo, hi).
// Two safeguards.  The Krylov basis behind G is close to linearly dependent
// and G, h are known only to a relative accuracy e (FP32 vectors), so the
// monomial form can report a small or even negative loss for large c; the
// objective is the loss plus its uncertainty e (2 |c|.|h| + |c|.|G| |c|).
// And hi covers the largest eigenvalue modulus of D^-1 L as the Gram data
// estimate it by power iteration, |y_8| / |y_7| with y_j = L (D^-1 L)^j D^-1 r
// (a residual polynomial above 1 in modulus past hi would make the
// preconditioned operator indefinite).  Host code only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bt_internal.h"

namespace {

// coefficients (in l, ascending) of r(l) for the interval [lo, hi]
void residual_poly(double lo, double hi, double r[10]) {
  const double a = (hi + lo) / (hi - lo), b = -2.0 / (hi - lo);  // x = a + b l
  double t0[10] = {1.0}, t1[10] = {a, b}, t2[10];
  for (int k = 1; k < 9; ++k) {  // t1 = T_k(x(l)), t0 = T_{k-1}
    for (int i = 0; i < 10; ++i) t2[i] = -t0[i];
    for (int i = 0; i + 1 < 10; ++i) {
      t2[i] += 2.0 * a * t1[i];
      t2[i + 1] += 2.0 * b * t1[i];
    }
    std::copy(t1, t1 + 10, t0);
    std::copy(t2, t2 + 10, t1);
  }
  for (int i = 0; i < 10; ++i) r[i] = t1[i] / t1[0];  // t1[0] = T_9(a) = r's value at l = 0
}

double mean_loss(const double* Gm, const double* hm, const double* c) {
  double v = 1.0;
  for (int i = 0; i < 9; ++i) {
    v -= 2.0 * c[i] * hm[i];
    for (int j = 0; j < 9; ++j) v += c[i] * Gm[9 * i + j] * c[j];
  }
  return v;
}

// the loss's uncertainty from data known to relative accuracy e
double loss_spread(const double* Ga, const double* ha, const double* c, double e) {
  double v = 0.0;
  for (int i = 0; i < 9; ++i) {
    v += 2.0 * std::fabs(c[i]) * ha[i];
    for (int j = 0; j < 9; ++j) v += std::fabs(c[i]) * Ga[9 * i + j] * std::fabs(c[j]);
  }
  return e * v;
}

}  // namespace

extern "C" bt_status bt_chebyshev_poly(double lo, double hi, double* c9) {
  if (!c9 || !(lo > 0) || !(hi > lo) || !std::isfinite(hi)) return BT_EINVAL;
  double r[10];
  residual_poly(lo, hi, r);
  for (int j = 0; j < 9; ++j) c9[j] = -r[j + 1];
  for (int j = 0; j < 9; ++j)
    if (!std::isfinite(c9[j])) return BT_EINVAL;
  return BT_OK;
}

extern "C" bt_status bt_fit_chebyshev(int64_t n, const double* G, const double* h, double rel_err, double* lo,
                                      double* hi, double* c9, double* loss) {
  if (n < 1 || !G || !h || !(rel_err >= 0) || !(rel_err < 1)) return BT_EINVAL;
  std::vector<double> Gm(81, 0.0), hm(9, 0.0), Ga(81, 0.0), ha(9, 0.0);
  double lam = 0.0;  // power-iteration estimate of max |eig(D^-1 L)| over the samples
  for (int64_t s = 0; s < n; ++s) {
    for (int i = 0; i < 81; ++i) Gm[i] += G[81 * s + i], Ga[i] += std::fabs(G[81 * s + i]);
    for (int i = 0; i < 9; ++i) hm[i] += h[9 * s + i], ha[i] += std::fabs(h[9 * s + i]);
    const double g77 = G[81 * s + 70], g88 = G[81 * s + 80];
    if (g77 > 0 && g88 > 0) lam = std::max(lam, std::sqrt(g88 / g77));
  }
  for (int i = 0; i < 81; ++i) Gm[i] /= (double)n, Ga[i] /= (double)n;
  for (int i = 0; i < 9; ++i) hm[i] /= (double)n, ha[i] /= (double)n;
  for (int i = 0; i < 81; ++i)
    if (!std::isfinite(Gm[i]) || !std::isfinite(Ga[i])) return BT_EINVAL;
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(hm[i]) || !std::isfinite(ha[i])) return BT_EINVAL;
  if (!std::isfinite(lam)) return BT_EINVAL;
  // log-spaced search over hi in [max(1/4, 1.05 lam), max(16, 4 lam)] and
  // lo/hi in [1e-4, 0.95], then three zooms around the best point, each a
  // quarter of the previous span (hi never below its floor)
  const double hfloor = std::max(0.25, 1.05 * lam);
  double best = INFINITY, bval = 0, blo = 0, bhi = 0, c[9];
  double lh0 = std::log(hfloor), lh1 = std::log(std::max(16.0, 4.0 * hfloor)), lr0 = std::log(1e-4),
         lr1 = std::log(0.95);
  const int M = 48;
  for (int zoom = 0; zoom < 4; ++zoom) {
    double cl = blo, ch = bhi;
    for (int i = 0; i <= M; ++i)
      for (int k = 0; k <= M; ++k) {
        const double H = std::exp(std::max(lh0 + (lh1 - lh0) * i / M, std::log(hfloor)));
        const double Lo = H * std::exp(std::min(lr0 + (lr1 - lr0) * k / M, std::log(0.95)));
        if (bt_chebyshev_poly(Lo, H, c) != BT_OK) continue;
        const double v = mean_loss(Gm.data(), hm.data(), c);
        const double obj = v + loss_spread(Ga.data(), ha.data(), c, rel_err);
        if (std::isfinite(obj) && obj < best) best = obj, bval = v, cl = Lo, ch = H;
      }
    blo = cl;
    bhi = ch;
    if (!(best < INFINITY)) return BT_EINVAL;
    const double sh = (lh1 - lh0) / 8.0, sr = (lr1 - lr0) / 8.0;
    const double ch_l = std::log(bhi), cr_l = std::log(blo / bhi);
    lh0 = ch_l - sh, lh1 = ch_l + sh, lr0 = cr_l - sr, lr1 = cr_l + sr;
  }
  if (lo) *lo = blo;
  if (hi) *hi = bhi;
  if (c9) bt_chebyshev_poly(blo, bhi, c9);
  if (loss) *loss = bval;
  return BT_OK;
}
