// Host FP64 thermodynamics for set-up: critical point and Maxwell
// coexistence densities of the van der Waals (Eq. 30) and Carnahan-Starling
// equations of state, written as mu(rho) = R T h(rho) - 2 a rho and
// p(rho) = rho mu(rho) - E_f(rho).
//
// Critical point: the spinodal temperature 2a / (R h'(rho)) peaks where
// h''(rho) = 0 (bisection). Maxwell construction (Sec. IV A): for a trial
// chemical potential m between the spinodal values, the gas and liquid
// branches give rho_g(m) < rho_l(m); bisection on m makes their pressures
// equal, then Newton on the 2x2 system polishes the pair.
#include <cmath>

#include "../../include/lbfe.h"

namespace {

struct Eos {
    int kind;
    double a, b, R;
    double rho_max() const { return kind == LB_VDW ? 1.0 / b : 4.0 / b; }
    double h(double r) const
    {
        if (kind == LB_VDW) {
            const double q = 1.0 / (1.0 - b * r);
            return std::log(r * q) + q;
        }
        const double n = 0.25 * b * r, q = 1.0 / (1.0 - n);
        return std::log(r) + 1.0 + n * (4.0 - 3.0 * n) * q * q + n * (4.0 - 2.0 * n) * q * q * q;
    }
    double dh(double r) const
    {
        if (kind == LB_VDW) {
            const double q = 1.0 / (1.0 - b * r);
            return 1.0 / r + b * q + b * q * q;
        }
        const double n = 0.25 * b * r, q = 1.0 / (1.0 - n);
        return 1.0 / r + 0.25 * b * (8.0 - 2.0 * n) * q * q * q * q;
    }
    double d2h(double r) const
    {
        if (kind == LB_VDW) {
            const double q = 1.0 / (1.0 - b * r);
            return -1.0 / (r * r) + b * b * q * q + 2.0 * b * b * q * q * q;
        }
        const double n = 0.25 * b * r, q = 1.0 / (1.0 - n);
        return -1.0 / (r * r) + 0.0625 * b * b * (30.0 - 6.0 * n) * q * q * q * q * q;
    }
    // free energy without the kappa term, for the pressure
    double Ef(double r, double T) const
    {
        if (kind == LB_VDW) return r * R * T * std::log(r / (1.0 - b * r)) - a * r * r;
        const double n = 0.25 * b * r, q = 1.0 / (1.0 - n);
        return R * T * r * std::log(r) + R * T * r * n * (4.0 - 3.0 * n) * q * q - a * r * r;
    }
    double mu(double r, double T) const { return R * T * h(r) - 2.0 * a * r; }
    double dmu(double r, double T) const { return R * T * dh(r) - 2.0 * a; }
    double p(double r, double T) const { return r * mu(r, T) - Ef(r, T); }
};

bool valid(int kind, double a, double b, double R)
{
    return (kind == LB_VDW || kind == LB_CS) && a > 0 && b > 0 && R > 0 && std::isfinite(a) &&
           std::isfinite(b) && std::isfinite(R);
}

double critical_rho(const Eos& e)
{
    double lo = 1e-9 * e.rho_max(), hi = (1.0 - 1e-9) * e.rho_max();
    for (int k = 0; k < 300; ++k) {
        const double m = 0.5 * (lo + hi);
        if (e.d2h(m) < 0.0) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
}

// root of g on (lo, hi) with g(lo) and g(hi) of opposite signs; geometric
// midpoints when the bracket spans decades
template <class G>
double bisect(G g, double lo, double hi)
{
    double glo = g(lo);
    for (int k = 0; k < 400; ++k) {
        const double m = (hi / lo > 4.0) ? std::sqrt(lo * hi) : 0.5 * (lo + hi);
        if (m <= lo || m >= hi) break;
        const double gm = g(m);
        if ((gm < 0.0) == (glo < 0.0)) { lo = m; glo = gm; } else hi = m;
    }
    return 0.5 * (lo + hi);
}

// spinodal densities s1 < rho_c < s2 at T < T_c (roots of mu'(rho) = 0)
void spinodals(const Eos& e, double T, double rc, double* s1, double* s2)
{
    const double target = 2.0 * e.a / (e.R * T);  // h'(rho) on the spinodal
    const double rmax = e.rho_max();
    // h' decreases to its minimum at rc, then increases
    double lo = rc;
    while (e.dh(lo) < target) lo *= 0.5;
    *s1 = bisect([&](double r) { return e.dh(r) - target; }, lo, rc);
    double hi = rc;
    while (e.dh(hi) < target) hi = 0.5 * (hi + rmax);
    *s2 = bisect([&](double r) { return e.dh(r) - target; }, rc, hi);
}

}  // namespace

extern "C" lb_status lb_critical(int32_t eos, double a, double b, double R, double* Tc, double* rho_c)
{
    if (!valid(eos, a, b, R) || !Tc || !rho_c) return LB_E_INVALID;
    const Eos e{eos, a, b, R};
    const double rc = critical_rho(e);
    *rho_c = rc;
    *Tc = 2.0 * a / (R * e.dh(rc));
    return LB_OK;
}

extern "C" lb_status lb_maxwell(int32_t eos, double a, double b, double R, double T, double* rho_g,
                                double* rho_l)
{
    if (!valid(eos, a, b, R) || !rho_g || !rho_l || !(T > 0)) return LB_E_INVALID;
    const Eos e{eos, a, b, R};
    const double rc = critical_rho(e);
    const double Tc = 2.0 * a / (R * e.dh(rc));
    if (!(T < Tc)) return LB_E_INVALID;
    const double rmax = e.rho_max();
    double s1, s2;
    spinodals(e, T, rc, &s1, &s2);
    const double mu_lo = e.mu(s2, T), mu_hi = e.mu(s1, T);
    auto gas = [&](double m) {
        double l = s1;
        while (e.mu(l, T) > m) l *= 0.5;
        return bisect([&](double r) { return e.mu(r, T) - m; }, l, s1);
    };
    auto liq = [&](double m) {
        double u = s2;
        while (e.mu(u, T) < m) u = 0.5 * (u + rmax);
        return bisect([&](double r) { return e.mu(r, T) - m; }, s2, u);
    };
    // d(p_l - p_g)/dm = rho_l - rho_g > 0 (Gibbs-Duhem): p_l - p_g rises from
    // < 0 to > 0 as m crosses (mu(s2), mu(s1))
    double ml = mu_lo, mh = mu_hi;
    for (int k = 0; k < 200; ++k) {
        const double m = 0.5 * (ml + mh);
        if (m <= ml || m >= mh) break;
        const double d = e.p(liq(m), T) - e.p(gas(m), T);
        if (d > 0.0) mh = m; else ml = m;
    }
    const double m = 0.5 * (ml + mh);
    double g = gas(m), l = liq(m);
    for (int k = 0; k < 20; ++k) {  // Newton polish
        const double f1 = e.p(g, T) - e.p(l, T), f2 = e.mu(g, T) - e.mu(l, T);
        const double dg = e.dmu(g, T), dl = e.dmu(l, T);
        const double j11 = g * dg, j12 = -l * dl, j21 = dg, j22 = -dl;
        const double det = j11 * j22 - j12 * j21;
        if (det == 0.0 || !std::isfinite(det)) break;
        const double d1 = (f1 * j22 - j12 * f2) / det, d2 = (j11 * f2 - j21 * f1) / det;
        if (!(g - d1 > 0.0) || !(l - d2 > 0.0)) break;
        g -= d1;
        l -= d2;
        if (std::fabs(d1) <= 1e-16 * g && std::fabs(d2) <= 1e-16 * l) break;
    }
    *rho_g = g;
    *rho_l = l;
    return LB_OK;
}

// Flat-interface tension of the square-gradient free energy (Eq. 1):
// sigma = int_{rho_g}^{rho_l} sqrt(2 kappa (E_f - mu rho + p)) drho at the
// Maxwell coexistence, by composite 5-point Gauss-Legendre quadrature over
// 4096 panels (the integrand vanishes linearly at both ends).
extern "C" lb_status lb_surface_tension(int32_t eos, double a, double b, double R, double T, double kappa,
                                        double* sigma)
{
    if (!sigma || !(kappa > 0) || !std::isfinite(kappa)) return LB_E_INVALID;
    double g, l;
    const lb_status s = lb_maxwell(eos, a, b, R, T, &g, &l);
    if (s != LB_OK) return s;
    const Eos e{eos, a, b, R};
    const double mu = e.mu(g, T), p = e.p(g, T);
    auto f = [&](double r) {
        const double w = e.Ef(r, T) - mu * r + p;
        return w > 0.0 ? std::sqrt(2.0 * kappa * w) : 0.0;
    };
    // 5-point Gauss-Legendre nodes and weights on [-1, 1]
    const double x[5] = {0.0, 0.5384693101056831, -0.5384693101056831, 0.9061798459386640, -0.9061798459386640};
    const double w[5] = {0.5688888888888889, 0.4786286704993665, 0.4786286704993665, 0.2369268850561891,
                         0.2369268850561891};
    constexpr int kPanels = 4096;
    const double hw = 0.5 * (l - g) / kPanels;
    double sum = 0.0;
    for (int k = 0; k < kPanels; ++k) {
        const double c = g + (2 * k + 1) * hw;
        double ps = 0.0;
        for (int q = 0; q < 5; ++q) ps += w[q] * f(c + hw * x[q]);
        sum += ps * hw;
    }
    *sigma = sum;
    return LB_OK;
}

// Eq. 32: the phase pressures around a circular droplet of radius r,
// p_sat + rho_sat / (rho_l_sat - rho_g_sat) sigma / r, each turned back into
// a density on its own branch of p_EOS (increasing on (rho_g_sat, s1) and
// above s2) by bisection.
extern "C" lb_status lb_young_laplace(int32_t eos, double a, double b, double R, double T, double sigma,
                                      double r, double* rho_g, double* rho_l)
{
    if (!rho_g || !rho_l || !(sigma >= 0) || !(r > 0) || !std::isfinite(sigma) || !std::isfinite(r))
        return LB_E_INVALID;
    double g, l;
    const lb_status s = lb_maxwell(eos, a, b, R, T, &g, &l);
    if (s != LB_OK) return s;
    const Eos e{eos, a, b, R};
    const double rc = critical_rho(e);
    double s1, s2;
    spinodals(e, T, rc, &s1, &s2);
    const double p0 = e.p(g, T);
    const double pl = p0 + l / (l - g) * sigma / r, pg = p0 + g / (l - g) * sigma / r;
    if (!(e.p(s1, T) > pg)) return LB_E_INVALID;  // droplet too small: no gas state at that pressure
    *rho_g = bisect([&](double q) { return e.p(q, T) - pg; }, g, s1);
    double hi = s2;
    while (e.p(hi, T) < pl) hi = 0.5 * (hi + e.rho_max());
    *rho_l = bisect([&](double q) { return e.p(q, T) - pl; }, s2, hi);
    return LB_OK;
}
