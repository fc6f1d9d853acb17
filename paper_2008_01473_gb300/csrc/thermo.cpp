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
    const double target = 2.0 * a / (R * T);  // h'(rho) on the spinodal
    const double rmax = e.rho_max();
    // spinodals: h' decreases to its minimum at rc, then increases
    double lo = rc;
    while (e.dh(lo) < target) lo *= 0.5;
    const double s1 = bisect([&](double r) { return e.dh(r) - target; }, lo, rc);
    double hi = rc;
    while (e.dh(hi) < target) hi = 0.5 * (hi + rmax);
    const double s2 = bisect([&](double r) { return e.dh(r) - target; }, rc, hi);
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
