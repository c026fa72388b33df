// Temporal profiles f(t) of the diffusion-encoding gradient: the tables the
// time loop needs, F(t_n) = int_0^{t_n} f on the time grid and int_0^TE F^2
// (b = q^2 int F^2, Section 2 Eq. b_value).  The paper's framework takes any
// profile (Section 3, "General diffusion-encoding sequence") and shows six of
// them (Section 4):
//   PGSE              f = +1 on [0, delta], -1 on [Delta, Delta + delta]
//   double PGSE       two PGSE blocks, the second starting at Delta + delta
//   cos-OGSE          f = cos(w s) on [0, delta], -cos(w (s - tau)) on
//                     (tau, tau + delta], w = 2 pi n / delta, tau = (delta + Delta)/2
//   sin-OGSE          the same with sin
//   trapezoidal PGSE  PGSE lobes with linear ramps of length `ramp` at both ends
//   double trapezoid  two trapezoid blocks, the second starting at Delta + delta
// F is written in closed form per profile; int F^2 is integrated with
// composite Gauss-Legendre quadrature between the profile's breakpoints (F is
// a polynomial or trigonometric function between them, so the quadrature is
// exact to rounding for the polynomial pieces and converges spectrally for
// the trigonometric ones).  Times in us.  Host code only.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bt_internal.h"

namespace {

double clampd(double x, double lo, double hi) { return std::min(std::max(x, lo), hi); }

// int_0^x of one lobe: the rectangle of length delta, or the trapezoid that
// rises over `ramp`, stays at 1 and falls over `ramp`
double lobe_rect(double x, double delta) { return clampd(x, 0.0, delta); }
double lobe_trap(double x, double delta, double r) {
  x = clampd(x, 0.0, delta);
  if (x <= r) return x * x / (2.0 * r);
  if (x <= delta - r) return r / 2.0 + (x - r);
  return delta - r - (delta - x) * (delta - x) / (2.0 * r);
}

struct Wave {
  int kind;
  double delta, Delta, w, tau, ramp;
  // F(t) = int_0^t f
  double F(double t) const {
    switch (kind) {
      case BT_PGSE:
        return lobe_rect(t, delta) - lobe_rect(t - Delta, delta);
      case BT_DOUBLE_PGSE: {
        const double T1 = Delta + delta;
        return lobe_rect(t, delta) - lobe_rect(t - Delta, delta) + lobe_rect(t - T1, delta) -
               lobe_rect(t - T1 - Delta, delta);
      }
      case BT_COS_OGSE:
      case BT_SIN_OGSE: {
        // antiderivative of the lobe shape from 0 to x in [0, delta]
        auto S = [&](double x) {
          x = clampd(x, 0.0, delta);
          return kind == BT_COS_OGSE ? std::sin(w * x) / w : (1.0 - std::cos(w * x)) / w;
        };
        return S(t) - S(t - tau);
      }
      case BT_TRAPEZOID:
        return lobe_trap(t, delta, ramp) - lobe_trap(t - Delta, delta, ramp);
      case BT_DOUBLE_TRAPEZOID: {
        const double T1 = Delta + delta;
        return lobe_trap(t, delta, ramp) - lobe_trap(t - Delta, delta, ramp) + lobe_trap(t - T1, delta, ramp) -
               lobe_trap(t - T1 - Delta, delta, ramp);
      }
    }
    return 0.0;
  }
  // end of the waveform (f = 0 afterwards)
  double end() const {
    switch (kind) {
      case BT_DOUBLE_PGSE:
      case BT_DOUBLE_TRAPEZOID:
        return 2.0 * (Delta + delta);
      case BT_COS_OGSE:
      case BT_SIN_OGSE:
        return tau + delta;
      default:
        return Delta + delta;
    }
  }
  // times where f is not smooth
  std::vector<double> breaks(double TE) const {
    std::vector<double> b{0.0, TE};
    std::vector<double> starts;
    if (kind == BT_COS_OGSE || kind == BT_SIN_OGSE) {
      for (double s : {0.0, delta, tau, tau + delta}) b.push_back(s);
    } else {
      starts = {0.0, Delta};
      if (kind == BT_DOUBLE_PGSE || kind == BT_DOUBLE_TRAPEZOID) {
        starts.push_back(Delta + delta);
        starts.push_back(2.0 * Delta + delta);
      }
      const double r = (kind == BT_TRAPEZOID || kind == BT_DOUBLE_TRAPEZOID) ? ramp : 0.0;
      for (double s0 : starts)
        for (double s : {s0, s0 + r, s0 + delta - r, s0 + delta}) b.push_back(s);
    }
    std::vector<double> out;
    for (double x : b)
      if (x >= 0.0 && x <= TE) out.push_back(x);
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
  }
};

// Gauss-Legendre nodes and weights on [-1, 1]: the roots of P_m by Newton's
// method on the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},
// with P_m' = m (x P_m - P_{m-1}) / (x^2 - 1) and w = 2 / ((1 - x^2) P_m'^2).
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (m + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < m; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[m - 1 - i] = z;
    w[i] = w[m - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

extern "C" bt_status bt_waveform_tables(int kind, double delta, double Delta, double TE, double dt,
                                        int32_t n_periods, double ramp, int32_t* n_steps, double* F,
                                        double* int_F2) {
  if (kind < BT_PGSE || kind > BT_DOUBLE_TRAPEZOID) return BT_EINVAL;
  if (!(delta > 0) || !(Delta >= delta) || !(dt > 0) || !(TE > 0) || !std::isfinite(TE)) return BT_EINVAL;
  Wave wv{kind, delta, Delta, 0.0, 0.5 * (delta + Delta), 0.0};
  if (kind == BT_COS_OGSE || kind == BT_SIN_OGSE) {
    if (n_periods < 1) return BT_EINVAL;
    wv.w = 2.0 * 3.14159265358979323846 * n_periods / delta;
  }
  if (kind == BT_TRAPEZOID || kind == BT_DOUBLE_TRAPEZOID) {
    wv.ramp = ramp > 0 ? ramp : delta / 10.0;
    if (wv.ramp > 0.5 * delta) return BT_EINVAL;
  }
  const double ns = TE / dt;
  const long long N = std::llround(ns);
  if (N < 1 || N > (1 << 24) || std::fabs(ns - (double)N) > 1e-9 * std::max(1.0, ns)) return BT_EINVAL;
  if (TE < wv.end() - 1e-9 * TE) return BT_EINVAL;
  if (n_steps) *n_steps = (int32_t)N;
  if (F) {
    for (long long n = 0; n <= N; ++n) F[n] = n == 0 ? 0.0 : wv.F((double)n * dt);
  }
  if (int_F2) {
    std::vector<double> gx, gw;
    gauss_legendre(10, gx, gw);
    const std::vector<double> bp = wv.breaks(TE);
    const int pieces = 64;
    double total = 0.0;
    for (size_t k = 0; k + 1 < bp.size(); ++k) {
      const double a = bp[k], b = bp[k + 1];
      if (!(b > a)) continue;
      for (int j = 0; j < pieces; ++j) {
        const double lo = a + (b - a) * j / pieces, hi = a + (b - a) * (j + 1) / pieces;
        const double c = 0.5 * (hi + lo), hw = 0.5 * (hi - lo);
        double s = 0.0;
        for (size_t i = 0; i < gx.size(); ++i) {
          const double f = wv.F(c + hw * gx[i]);
          s += gw[i] * f * f;
        }
        total += hw * s;
      }
    }
    *int_F2 = total;
  }
  return BT_OK;
}
