// Host-side construction of the C1 sum-of-Gaussians decomposition of the Yukawa
// kernel Y(r) = exp(-r/lambda)/r (Algorithm 1), in FP64.
//
//   f(t,r) = pi^{-1/2} exp(-r^2 e^t - 1/(4 lambda^2 e^t) + t/2)                 Eq. (1)
//   h      = pi^2 / (log(eps + 6 sqrt(2 pi) e^{1/6}/r_c) + log(1/eps))          Eq. (27)
//   F(r)   = h [ w f(t_M2, r) + sum_{m=-M1}^{M2-1} f(t_m, r) ]                  Eq. (37)
//   w      from the C0 condition Y(r_c) = F(r_c)                                Eq. (38)
//   t0     smallest root in [0, h) of the C1 condition d/dr[Y - F](r_c) = 0     Eq. (36)
//   M1, M2 "bound" mode: ceilings of Eqs. (29)-(30) at alpha_1 of Eq. (35);
//          "minimal" mode: the fewest Gaussians with max |Y - F| <= eps on a
//          2000-point logarithmic grid of [r_c, 33 lambda] (R = 33 lambda, Sec. 3.2),
//          ties broken by the smaller error.
// Roots of the C1 residual are bracketed on a 200-interval grid over [0, h] and
// refined by bisection to the last bit.  The Lambert W of Eq. (29) is computed by
// Halley's iteration on w e^w = x.
#include "sog_host.h"

#include <cmath>
#include <cstdio>
#include <vector>

namespace rbsog {

namespace {
const double kPi = 3.14159265358979323846;
const double kInvSqrtPi = 0.56418958354775628695;
const int kErrGrid = 2000;
const int kRootGrid = 200;

double yukawa(double r, double lam) { return std::exp(-r / lam) / r; }
double dyukawa(double r, double lam) { return -std::exp(-r / lam) * (1.0 / (lam * r) + 1.0 / (r * r)); }

double step_h(double eps, double delta) {
    return kPi * kPi / (std::log(eps + 6.0 * std::sqrt(2.0 * kPi) * std::exp(1.0 / 6.0) / delta) + std::log(1.0 / eps));
}

double posmod(double x, double h) { return x - h * std::floor(x / h); }

// principal branch of Lambert W for x > 0 (Halley's method)
double lambert_w0(double x) {
    double w = x < 2.718281828459045 ? std::log1p(x) * 0.8 : std::log(x) - std::log(std::log(x));
    for (int it = 0; it < 100; ++it) {
        double ew = std::exp(w);
        double f = w * ew - x;
        double wp1 = w + 1.0;
        double dw = f / (ew * wp1 - (w + 2.0) * f / (2.0 * wp1));
        w -= dw;
        if (std::fabs(dw) <= 1e-15 * (1.0 + std::fabs(w))) break;
    }
    return w;
}

// C0 weight of Eq. (38); NaN when the narrowest Gaussian underflows at r_c
double c0_weight(double t0, double h, int M1, int M2, double lam, double rc) {
    double partial = 0.0;
    for (int m = -M1; m < M2; ++m) partial += sog_f(t0 + m * h, rc, lam);
    partial *= h;
    double den = h * sog_f(t0 + M2 * h, rc, lam);
    if (!(den > 0.0)) return NAN;
    return (yukawa(rc, lam) - partial) / den;
}

// C1 residual of Eq. (36) with the C0 weight
double c1_residual(double t0, double h, int M1, int M2, double lam, double rc) {
    double w = c0_weight(t0, h, M1, M2, lam, rc);
    if (!std::isfinite(w)) return NAN;
    double dF = 0.0;
    for (int m = -M1; m <= M2; ++m) {
        double t = t0 + m * h;
        double wt = (m == M2) ? w : 1.0;
        dF += wt * (-2.0 * rc * std::exp(t)) * sog_f(t, rc, lam);
    }
    return dyukawa(rc, lam) - h * dF;
}

bool smallest_c1_root(double h, int M1, int M2, double lam, double rc, double *t0) {
    double prev_x = 0.0, prev_v = c1_residual(0.0, h, M1, M2, lam, rc);
    for (int k = 1; k <= kRootGrid; ++k) {
        double x = h * (double)k / (double)kRootGrid;
        double v = c1_residual(x, h, M1, M2, lam, rc);
        if (std::isfinite(prev_v) && std::isfinite(v)) {
            if (prev_v == 0.0) { *t0 = prev_x; return true; }
            if ((prev_v < 0.0) != (v < 0.0) && v != 0.0) {
                double a = prev_x, b = x, fa = prev_v;
                for (int it = 0; it < 200; ++it) {
                    double mid = 0.5 * (a + b);
                    if (mid <= a || mid >= b) break;
                    double fm = c1_residual(mid, h, M1, M2, lam, rc);
                    if (!std::isfinite(fm) || fm == 0.0) { a = b = mid; break; }
                    if ((fm < 0.0) == (fa < 0.0)) { a = mid; fa = fm; } else { b = mid; }
                }
                double r = 0.5 * (a + b);
                if (r < h) { *t0 = r; return true; }
            }
        }
        prev_x = x;
        prev_v = v;
    }
    return false;
}

bool build_table(double lam, double rc, double eps, int M1, int M2, SogDecomp *s) {
    if (M1 + M2 + 1 < 1) return false;
    double h = step_h(eps, rc);
    double t0;
    if (!smallest_c1_root(h, M1, M2, lam, rc, &t0)) return false;
    s->lam = lam; s->rc = rc; s->eps = eps; s->h = h; s->t0 = t0; s->M1 = M1; s->M2 = M2;
    s->w = c0_weight(t0, h, M1, M2, lam, rc);
    return std::isfinite(s->w);
}

double m1_bound(double t0, double h, double lam, double eps) {
    return (t0 - std::log(kPi * eps * eps / 36.0) - lambert_w0(18.0 / (kPi * lam * lam * eps * eps))) / h;
}

double m2_bound(double t0, double h, double eps, double delta, double R) {
    double a = -t0 - 2.0 * std::log(delta) + std::log(std::log(3.0 / (eps * delta)));
    double b = -t0 - h - 2.0 * std::log(std::sqrt(2.0) * R);
    return (a > b ? a : b) / h;
}

double alpha1(double h, double lam, double rc) {
    double base = -std::log(2.0 * lam * rc);
    double a = posmod(base + h / 4.0, h), b = posmod(base + 3.0 * h / 4.0, h);
    return a < b ? a : b;
}
}  // namespace

double sog_f(double t, double r, double lam) {
    double et = std::exp(t);
    return std::exp(-r * r * et - 1.0 / (4.0 * lam * lam * et) + 0.5 * t) * kInvSqrtPi;
}

double sog_far(const SogDecomp &s, double r) {
    double acc = 0.0;
    for (int m = -s.M1; m <= s.M2; ++m) acc += ((m == s.M2) ? s.w : 1.0) * sog_f(s.t0 + m * s.h, r, s.lam);
    return s.h * acc;
}

double sog_max_error(const SogDecomp &s) {
    // logarithmic grid with exact end points: r_i = 10^(log10 r_c + i (log10 R - log10 r_c)/(n-1))
    double R = 33.0 * s.lam;
    double a = std::log10(s.rc), b = std::log10(R), step = (b - a) / (double)(kErrGrid - 1);
    double worst = 0.0;
    for (int i = 0; i < kErrGrid; ++i) {
        double r = (i == 0) ? s.rc : (i == kErrGrid - 1) ? R : std::pow(10.0, (double)i * step + a);
        double e = std::fabs(yukawa(r, s.lam) - sog_far(s, r));
        if (!(e <= worst)) worst = e;
    }
    return worst;
}

bool build_sog(double lam, double rc, double eps, int mode, int M1, int M2, SogDecomp *out, std::string *err) {
    char buf[256];
    if (!(lam > 0) || !(rc > 0) || !(eps > 0 && eps <= 0.1)) {
        *err = "SOG: need lambda > 0, r_c > 0 and 0 < eps <= 0.1";
        return false;
    }
    if (mode == 2) {
        if (!build_table(lam, rc, eps, M1, M2, out)) {
            std::snprintf(buf, sizeof buf, "SOG: no C1 root in [0,h) for M1=%d M2=%d", M1, M2);
            *err = buf;
            return false;
        }
        return true;
    }
    double h = step_h(eps, rc);
    double a1 = alpha1(h, lam, rc);
    if (mode == 1) {
        int m1 = (int)std::ceil(m1_bound(a1, h, lam, eps));
        int m2 = (int)std::ceil(m2_bound(a1, h, eps, rc, 33.0 * lam));
        if (!build_table(lam, rc, eps, m1, m2, out)) {
            *err = "SOG: bound-mode (M1, M2) has no C1 root in [0,h)";
            return false;
        }
        return true;
    }
    int m2c = (int)std::ceil(m2_bound(a1, h, eps, rc, 33.0 * lam));
    for (int mtot = 1; mtot <= 40; ++mtot) {
        bool found = false;
        double best_err = 0.0;
        SogDecomp best;
        for (int m2 = m2c - mtot - 3; m2 <= m2c + 3; ++m2) {
            int m1 = mtot - 1 - m2;
            SogDecomp s;
            if (!build_table(lam, rc, eps, m1, m2, &s)) continue;
            double e = sog_max_error(s);
            if (e <= eps && (!found || e < best_err)) {
                found = true;
                best_err = e;
                best = s;
            }
        }
        if (found) {
            *out = best;
            return true;
        }
    }
    *err = "SOG: no decomposition with at most 40 Gaussians meets eps";
    return false;
}

}  // namespace rbsog
