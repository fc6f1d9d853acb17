"""The oracle's step, linearised about a uniform state at rest, against a
Fourier (von Neumann) analysis of the scheme written out here from the paper.

About a uniform density rho0 with u = 0, one step maps a perturbation
delta f(x) = Re(v exp(i k.x)) to Re(A(k) v exp(i k.x)) + O(|v|^2), where
A(k) follows from Eq. 10 (streaming: a phase exp(-i k.e_a) per direction),
Eq. 12 (rho, u with half the force), Eq. 2 with Eq. 30 (mu_c), the Eq. 17
gradient and the 9-point Laplacian as Fourier symbols, Eq. 13 or Eq. 24
(force), Eq. 11 or Eq. 27 (equilibrium moments), the forcing moments of
Eq. 14 at u = 0, Eq. 29 (correction) and Eq. 28 (moment-space collision).
Nothing below calls the oracle's arithmetic: the moment matrix, the
equilibria, the source and the stencils are restated in Fourier space.
A dropped term, a wrong sign or factor in C, S, m_eq or the force, or a
transposed stencil changes A(k) and fails the one-step comparison.

The growth test pins the finding that the improved scheme with the Eq. 17
discretisation of d(phi u) leaves the vapour at 0.7 T_c linearly unstable:
the oracle's perturbation grows at the spectral radius of A(k).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from oracle import thermo

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
# Lallemand-Luo moments (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy), written
# out row by row from their definitions in terms of e_a
_E2 = EX**2 + EY**2
MOM = np.array([np.ones(9), -4 + 3 * _E2, 4 - 10.5 * _E2 + 4.5 * _E2**2, EX, (3 * _E2 - 5) * EX, EY,
                (3 * _E2 - 5) * EY, EX**2 - EY**2, EX * EY], dtype=float)


def dmu0_vdw(rho, a, b, R, T):
    """d/drho of the bulk part of Eq. 30, RT[ln(rho/(1 - b rho)) + 1/(1 - b rho)] - 2 a rho."""
    return R * T * (1.0 / rho + b / (1.0 - b * rho) + b / (1.0 - b * rho) ** 2) - 2.0 * a


def mu0_vdw(rho, a, b, R, T):
    return R * T * (np.log(rho / (1.0 - b * rho)) + 1.0 / (1.0 - b * rho)) - 2.0 * a * rho


def amplification(case: O.Case, rho0: float, kx: float, ky: float, with_c: bool = True) -> np.ndarray:
    """A(k): the one-step map of population perturbations (pre-collision
    storage: collide, then stream) about (rho0, u = 0); with_c = False
    leaves out the correction of Eq. 28."""
    ph = np.exp(1j * (kx * EX + ky * EY))
    gx = 3.0 * np.sum(W * EX * ph)  # Eq. 17 symbol
    gy = 3.0 * np.sum(W * EY * ph)
    lap = 6.0 * np.sum(W * (ph - 1.0))  # 9-point Laplacian symbol
    T = case.T
    dmu_drho = dmu0_vdw(rho0, case.a, case.b, case.R, T) - case.kappa * lap
    pm3 = case.pm_c0 + mu0_vdw(rho0, case.a, case.b, case.R, T)  # 3 p_m at the base state
    phi0 = (rho0 - pm3) / 3.0
    if case.collision == O.BGK:
        lam = np.full(9, 1.0 / case.tau_v)
    else:
        lam = np.array([0.0, 1 / case.tau_e, 1 / case.tau_s, 1.0, 1 / case.tau_q, 1.0, 1 / case.tau_q,
                        1 / case.tau_v, 1 / case.tau_v])
    Minv = np.linalg.inv(MOM)
    A = np.zeros((9, 9), complex)
    for col in range(9):
        df = np.zeros(9, complex)
        df[col] = 1.0
        m = MOM @ df
        drho, jx, jy = m[0], m[3], m[5]
        dmu = dmu_drho * drho
        improved = case.scheme in (O.IMPROVED, O.IMPROVED_SMOOTH)
        if improved:
            Fx, Fy = (1 / 3 - rho0) * gx * dmu, (1 / 3 - rho0) * gy * dmu  # Eq. 24
        else:
            Fx, Fy = gx * drho / 3 - rho0 * gx * dmu, gy * drho / 3 - rho0 * gy * dmu  # Eq. 13
        ux, uy = (jx + Fx / 2) / rho0, (jy + Fy / 2) / rho0
        if improved:  # Eq. 27 to first order: rho gamma = 3 p_m
            q = pm3 - 2 * rho0
            meq = np.array([drho, -4 * drho + 2 * dmu, 4 * drho - 3 * dmu, rho0 * ux, q * ux, rho0 * uy, q * uy,
                            0, 0])
        else:  # Eq. 11
            meq = np.array([drho, -2 * drho, drho, rho0 * ux, -rho0 * ux, rho0 * uy, -rho0 * uy, 0, 0])
        S = np.array([0, 0, 0, Fx, -Fx, Fy, -Fy, 0, 0])  # moments of Eq. 14 at u = 0
        Cv = np.zeros(9, complex)
        if case.scheme in (O.IMPROVED, O.IMPROVED_SMOOTH) and with_c:  # Eq. 29 about u = 0: d(phi u) = phi0 du
            avg = np.sum(W * ph) if case.scheme == O.IMPROVED_SMOOTH else 1.0  # lattice-weight average
            Ax, By = gx * avg * phi0 * ux, gy * avg * phi0 * uy
            Cv[1], Cv[7] = 9 * (Ax + By), 3 * (Ax - By)
        ms = m - lam * (m - meq) + (1 - lam / 2) * (S + Cv)  # Eq. 28
        A[:, col] = np.conj(ph) * (Minv @ ms)  # pull streaming, Eq. 10
    return A


def _perturbed(case, rho0, kx_idx, ky_idx, eps, seed):
    f0 = O.init(case, np.full((case.ny, case.nx), rho0))
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    y, x = np.mgrid[0:case.ny, 0:case.nx]
    kx, ky = 2 * np.pi * kx_idx / case.nx, 2 * np.pi * ky_idx / case.ny
    wave = np.exp(1j * (kx * x + ky * y))
    df = eps * np.real(v[:, None, None] * wave[None])
    return f0, np.ascontiguousarray(f0 + df), v, wave, kx, ky


CASES = [
    # (scheme, collision, T/T_c, phase, extra case fields, (kx index, ky index), lattice)
    (O.IMPROVED, O.BGK, 0.8, "gas", dict(tau_v=0.8), (2, 0), (10, 5)),
    (O.IMPROVED, O.BGK, 0.8, "liquid", dict(tau_v=1.0), (1, 1), (10, 10)),
    (O.IMPROVED, O.MRT, 0.85, "gas", dict(tau_v=0.7, tau_e=0.9, tau_s=1.2, tau_q=1.1), (3, 2), (10, 10)),
    (O.IMPROVED, O.MRT, 0.7, "gas", dict(tau_v=1.0, tau_e=1.0, tau_s=1.0, tau_q=1.1), (4, 0), (10, 5)),
    (O.STANDARD, O.BGK, 0.8, "gas", dict(tau_v=0.9), (1, 2), (10, 10)),
    (O.STANDARD, O.MRT, 0.9, "liquid", dict(tau_v=0.8, tau_e=1.1, tau_s=0.9, tau_q=1.2), (4, 3), (10, 10)),
    (O.IMPROVED_SMOOTH, O.BGK, 0.8, "gas", dict(tau_v=0.9), (3, 1), (10, 10)),
    (O.IMPROVED_SMOOTH, O.MRT, 0.7, "liquid", dict(tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1), (2, 3), (10, 10)),
]


@pytest.mark.parametrize("scheme,coll,tr,phase,kw,kidx,shape", CASES)
def test_one_step_matches_the_fourier_analysis(scheme, coll, tr, phase, kw, kidx, shape):
    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, tr)
    rho0 = rg if phase == "gas" else rl
    nx, ny = shape
    c = O.Case(nx=nx, ny=ny, scheme=scheme, collision=coll, eos=O.VDW, a=e.a, b=e.b, R=1.0, T=T, kappa=0.02, **kw)
    eps = 1e-7
    f0, f, v, wave, kx, ky = _perturbed(c, rho0, kidx[0], kidx[1], eps, seed=kidx[0] + 7 * kidx[1])
    assert O.step(c, f, 1) == 1
    got = f - f0
    want = eps * np.real((amplification(c, rho0, kx, ky) @ v)[:, None, None] * wave[None])
    scale = np.abs(want).max()
    assert scale > 1e-9
    assert np.abs(got - want).max() < 1e-5 * scale


def test_uniform_vapour_at_0p7_tc_grows_at_the_spectral_radius():
    """Improved scheme, BGK tau 1, vdW vapour at 0.7 T_c: the mode of
    wavelength 2.5 nodes (k = 0.8 pi) is unstable; the oracle's perturbation
    grows at the largest |eigenvalue| of A(k), 1.0201 per step, and the same
    state without the correction C is neutrally stable."""
    e = thermo.vdw_paper()
    T, rg, _ = thermo.maxwell_reduced(e, 0.7)
    c = O.Case(nx=5, ny=3, scheme=O.IMPROVED, collision=O.BGK, eos=O.VDW, a=e.a, b=e.b, R=1.0, T=T, kappa=0.02,
               tau_v=1.0)
    k = 2 * np.pi * 2 / 5
    lam = np.abs(np.linalg.eigvals(amplification(c, rg, k, 0.0)))
    rho_max = lam.max()
    assert 1.015 < rho_max < 1.025
    f0, f, *_ = _perturbed(c, rg, 2, 0, 1e-12, seed=3)
    O.step(c, f, 200)
    n1 = np.linalg.norm(f - f0)
    O.step(c, f, 300)
    n2 = np.linalg.norm(f - f0)
    assert n2 < 1e-6  # still linear
    assert abs((n2 / n1) ** (1 / 300) - rho_max) < 2e-5
    lam_no = np.abs(np.linalg.eigvals(amplification(c, rg, k, 0.0, with_c=False)))
    assert lam_no.max() < 1.0 + 1e-12



@pytest.mark.parametrize("flag", [O.FLAG_DROP_C, O.FLAG_FLIP_HALF_FORCE])
def test_planted_mistakes_break_the_one_step_comparison(flag):
    """The oracle's planted-mistake flags (C dropped; the half force in u with
    the wrong sign) move the linearised step well outside the tolerance."""
    e = thermo.vdw_paper()
    T, rg, _ = thermo.maxwell_reduced(e, 0.8)
    c = O.Case(nx=10, ny=10, scheme=O.IMPROVED, collision=O.BGK, eos=O.VDW, a=e.a, b=e.b, R=1.0, T=T, kappa=0.02,
               tau_v=0.8, flags=flag)
    eps = 1e-7
    f0, f, v, wave, kx, ky = _perturbed(c, rg, 3, 1, eps, seed=11)
    O.step(c, f, 1)
    want = eps * np.real((amplification(c, rg, kx, ky) @ v)[:, None, None] * wave[None])
    assert np.abs((f - f0) - want).max() > 1e-3 * np.abs(want).max()


def test_smoothed_correction_keeps_the_0p7_tc_vapour_stable():
    """With Eq. 29's derivatives taken on the lattice-weight average of phi u
    (scheme 3), the 0.7 T_c vapour has no growing Fourier mode for BGK tau 0.8
    and 1 (axis and oblique wave vectors), nor with MRT at the constant
    kinematic viscosity 0.04 of Table II; the oracle's perturbation at
    k = 0.8 pi decays."""
    e = thermo.vdw_paper()
    T, rg, _ = thermo.maxwell_reduced(e, 0.7)
    ks = np.linspace(0.0, np.pi, 13)
    base = dict(nx=5, ny=3, scheme=O.IMPROVED_SMOOTH, eos=O.VDW, a=e.a, b=e.b, R=1.0, T=T, kappa=0.02)
    pm = (1.0 + mu0_vdw(rg, e.a, e.b, 1.0, T)) / 3.0
    for kw in (dict(collision=O.BGK, tau_v=0.8), dict(collision=O.BGK, tau_v=1.0),
               dict(collision=O.MRT, tau_v=0.5 + 0.04 * rg / pm, tau_e=1.0, tau_s=1.0, tau_q=1.1)):
        c = O.Case(**base, **kw)
        worst = max(np.abs(np.linalg.eigvals(amplification(c, rg, kx, ky))).max() for kx in ks for ky in ks)
        assert worst < 1.0 + 1e-12, (kw, worst)
    c = O.Case(**base, collision=O.BGK, tau_v=1.0)
    f0, f, *_ = _perturbed(c, rg, 2, 0, 1e-9, seed=3)
    O.step(c, f, 100)
    n1 = np.linalg.norm(f - f0)
    O.step(c, f, 300)
    assert np.linalg.norm(f - f0) < n1
