"""FP64 thermodynamics of the oracle: equations of state, critical point and
the Maxwell equal-area construction.

TEST INFRASTRUCTURE ONLY: the product path never imports this module.

* van der Waals: E_f(rho) = rho R T ln[rho/(1 - b rho)] - a rho^2, whose
  derivative is the bulk part of the chemical potential of Eq. 30; the paper
  gives rho_c = 1/(3b) and T_c = 8a/(27 R b) beside it.
* Carnahan-Starling (not in the paper; used by the synthetic workloads):
  E_f = RT rho ln rho + RT rho (4n - 3n^2)/(1 - n)^2 - a rho^2, n = b rho / 4,
  whose p_EOS = rho E_f' - E_f is the Carnahan-Starling pressure
  rho R T (1 + n + n^2 - n^3)/(1 - n)^3 - a rho^2.
* p_EOS = rho E_f'(rho) - E_f(rho), the non-ideal equation of state below Eq. 4.
* Maxwell construction (Sec. IV A, Table II): rho_g < rho_l with equal
  pressure and equal chemical potential.

Derivatives of mu are taken by complex-step differentiation, which is exact to
rounding for these analytic functions.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq, minimize_scalar

VDW = 0
CS = 1


@dataclass(frozen=True)
class EOS:
    kind: int  # VDW or CS
    a: float
    b: float
    R: float = 1.0

    @property
    def rho_max(self) -> float:
        """Upper end of the physical density range (1 - b rho > 0, or n < 1)."""
        return 1.0 / self.b if self.kind == VDW else 4.0 / self.b

    def h(self, rho):
        """mu = R T h(rho) - 2 a rho: the temperature-scaled part of E_f'."""
        if self.kind == VDW:
            om = 1.0 - self.b * rho
            return np.log(rho / om) + 1.0 / om
        n = self.b * rho / 4.0
        om = 1.0 - n
        return np.log(rho) + 1.0 + (4.0 * n - 3.0 * n * n) / om**2 + n * (4.0 - 2.0 * n) / om**3

    def Ef(self, rho, T):
        if self.kind == VDW:
            return rho * self.R * T * np.log(rho / (1.0 - self.b * rho)) - self.a * rho * rho
        n = self.b * rho / 4.0
        om = 1.0 - n
        return (self.R * T * rho * np.log(rho) + self.R * T * rho * (4.0 * n - 3.0 * n * n) / om**2
                - self.a * rho * rho)

    def mu(self, rho, T):
        """Bulk chemical potential E_f'(rho) (Eq. 2 without the kappa term)."""
        return self.R * T * self.h(rho) - 2.0 * self.a * rho

    def p(self, rho, T):
        """p_EOS = rho E_f' - E_f."""
        return rho * self.mu(rho, T) - self.Ef(rho, T)

    def dh(self, rho: float) -> float:
        """h'(rho) by complex step."""
        step = 1e-30
        return float(np.imag(self.h(complex(rho, step))) / step)

    def dmu(self, rho: float, T: float) -> float:
        return self.R * T * self.dh(rho) - 2.0 * self.a

    # -- critical point: the spinodal temperature T_s(rho) = 2a/(R h'(rho)) peaks at T_c.
    def critical(self) -> tuple[float, float]:
        """(T_c, rho_c) as the maximum of the spinodal curve."""
        hi = 0.999 * self.rho_max
        res = minimize_scalar(lambda r: self.dh(r), bounds=(1e-6 * hi, hi), method="bounded",
                              options={"xatol": 1e-13 * hi, "maxiter": 500})
        rho_c = float(res.x)
        return 2.0 * self.a / (self.R * self.dh(rho_c)), rho_c

    def spinodals(self, T: float) -> tuple[float, float]:
        """The two roots of mu'(rho) = 0 below T_c."""
        _, rho_c = self.critical()
        target = 2.0 * self.a / (self.R * T)  # h'(rho) = target on the spinodal
        g = lambda r: self.dh(r) - target
        lo = rho_c
        while g(lo) < 0.0 and lo > 1e-300:
            lo *= 0.5
        s1 = brentq(g, lo, rho_c, xtol=1e-15, rtol=1e-15)
        hi = rho_c
        top = self.rho_max
        while g(hi) < 0.0:
            hi = 0.5 * (hi + top)
        s2 = brentq(g, rho_c, hi, xtol=1e-15, rtol=1e-15)
        return s1, s2

    def maxwell(self, T: float) -> tuple[float, float]:
        """(rho_g, rho_l) of the Maxwell construction at absolute temperature T.

        Pressure bracketing between the spinodal pressures, then a 2x2 Newton
        polish of p(rho_g) = p(rho_l), mu(rho_g) = mu(rho_l).
        """
        s1, s2 = self.spinodals(T)
        p_hi = float(self.p(s1, T))
        p_lo = max(float(self.p(s2, T)), 1e-300)

        def rho_gas(P):
            lo = s1
            while self.p(lo, T) > P:
                lo *= 0.5
            return brentq(lambda r: self.p(r, T) - P, lo, s1, xtol=1e-300, rtol=1e-15)

        def rho_liq(P):
            hi = s2
            top = self.rho_max
            while self.p(hi, T) < P:
                hi = 0.5 * (hi + top)
            return brentq(lambda r: self.p(r, T) - P, s2, hi, xtol=1e-300, rtol=1e-15)

        def dmu_of_p(P):
            return float(self.mu(rho_liq(P), T) - self.mu(rho_gas(P), T))

        # dmu_of_p goes from > 0 near p_lo to < 0 near p_hi
        eps = 1e-12 * (p_hi - p_lo)
        P = brentq(dmu_of_p, p_lo + eps, p_hi - eps, xtol=1e-300, rtol=1e-15, maxiter=400)
        rg, rl = rho_gas(P), rho_liq(P)
        for _ in range(8):
            f1 = float(self.p(rg, T) - self.p(rl, T))
            f2 = float(self.mu(rg, T) - self.mu(rl, T))
            a11, a12 = rg * self.dmu(rg, T), -rl * self.dmu(rl, T)
            a21, a22 = self.dmu(rg, T), -self.dmu(rl, T)
            det = a11 * a22 - a12 * a21
            if det == 0.0:
                break
            d1 = (f1 * a22 - a12 * f2) / det
            d2 = (a11 * f2 - a21 * f1) / det
            rg, rl = rg - d1, rl - d2
            if abs(d1) <= 1e-16 * rg and abs(d2) <= 1e-16 * rl:
                break
        return float(rg), float(rl)


    def surface_tension(self, T: float, kappa: float) -> float:
        """Flat-interface tension of the square-gradient free energy (Eq. 1):
        sigma = int_{rho_g}^{rho_l} sqrt(2 kappa (E_f - mu rho + p)) drho at
        coexistence (Maxwell densities, their mu and p)."""
        from scipy.integrate import quad

        rg, rl = self.maxwell(T)
        mu, p = float(self.mu(rg, T)), float(self.p(rg, T))
        f = lambda r: np.sqrt(max(2.0 * kappa * float(self.Ef(r, T) - mu * r + p), 0.0))
        return float(quad(f, rg, rl, limit=400, epsabs=0.0, epsrel=1e-12)[0])

    def young_laplace(self, T: float, sigma: float, r: float) -> tuple[float, float]:
        """(rho_g, rho_l) around a circular droplet of radius r (Eq. 32): the
        phase pressures p_sat + rho_sat / (rho_l_sat - rho_g_sat) sigma / r,
        each inverted on its branch of p_EOS."""
        rg, rl = self.maxwell(T)
        p0 = float(self.p(rg, T))
        pl = p0 + rl / (rl - rg) * sigma / r
        pg = p0 + rg / (rl - rg) * sigma / r
        s1, s2 = self.spinodals(T)
        hi = s2
        while self.p(hi, T) < pl:
            hi = 0.5 * (hi + self.rho_max)
        g = brentq(lambda q: self.p(q, T) - pg, rg, s1, xtol=1e-300, rtol=1e-15)
        l = brentq(lambda q: self.p(q, T) - pl, s2, hi, xtol=1e-300, rtol=1e-15)
        return float(g), float(l)


# Parameter sets used with the paper's experiments and the synthetic workloads.
def vdw_paper() -> EOS:
    """Sec. IV A: a = 9/392, b = 2/21, R = 1 (kappa = 0.02)."""
    return EOS(VDW, 9.0 / 392.0, 2.0 / 21.0, 1.0)


def cs_unit() -> EOS:
    """Carnahan-Starling with a = 1, b = 4, R = 1."""
    return EOS(CS, 1.0, 4.0, 1.0)


def maxwell_reduced(eos: EOS, t_over_tc: float) -> tuple[float, float, float]:
    """(T, rho_g, rho_l) for a reduced temperature T/T_c."""
    tc, _ = eos.critical()
    T = t_over_tc * tc
    rg, rl = eos.maxwell(T)
    return T, rg, rl


__all__ = ["EOS", "VDW", "CS", "vdw_paper", "cs_unit", "maxwell_reduced"]
