"""Pins of the oracle's adjoint (reverse sweep of the literal step) against
central finite differences of the oracle's own forward loss, in FP64.

Loss: L = sum_{n >= u_from} sum_x |u^n|^2 + sum_x s(x) rho^N(x); parameters
kappa (Eq. 2), T (Eq. 30) and the initial density rho0. The sweep is rebuilt
from checkpoints, so the 27-step runs also cover segment boundaries."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from oracle import thermo
from paper_2008_01473_gb300 import inputs


def _setup(scheme, collision, flags=0):
    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, 0.8)
    c = O.Case(nx=12, ny=10, scheme=scheme, collision=collision, eos=O.VDW, a=e.a, b=e.b, T=T, kappa=0.02,
               tau_v=0.8, flags=flags)
    rho0 = inputs.droplet(12, 10, 3.0, rl, rg, width=3.0, noise=1e-3, seed=1)
    sf = 1e-3 * (2 * inputs.splitmix_uniform(5, 0, 12, 10) - 1)
    return c, rho0, sf


N, U_FROM = 27, 15


def _fd(c, rho0, sf, which, h, v=None):
    if which == "kappa":
        return (O.loss(dataclasses.replace(c, kappa=c.kappa + h), rho0, N, U_FROM, sf)
                - O.loss(dataclasses.replace(c, kappa=c.kappa - h), rho0, N, U_FROM, sf)) / (2 * h)
    if which == "T":
        return (O.loss(dataclasses.replace(c, T=c.T + h), rho0, N, U_FROM, sf)
                - O.loss(dataclasses.replace(c, T=c.T - h), rho0, N, U_FROM, sf)) / (2 * h)
    return (O.loss(c, rho0 + h * v, N, U_FROM, sf) - O.loss(c, rho0 - h * v, N, U_FROM, sf)) / (2 * h)


@pytest.mark.parametrize("scheme", [O.STANDARD, O.IMPROVED])
@pytest.mark.parametrize("collision", [O.BGK, O.MRT])
def test_adjoint_matches_central_differences(scheme, collision):
    c, rho0, sf = _setup(scheme, collision)
    L, g, gk, gT = O.adjoint(c, rho0, N, U_FROM, sf)
    assert abs(L / O.loss(c, rho0, N, U_FROM, sf) - 1) < 1e-13
    assert abs(gk / _fd(c, rho0, sf, "kappa", 1e-6) - 1) < 1e-6
    assert abs(gT / _fd(c, rho0, sf, "T", 1e-6 * c.T) - 1) < 1e-6
    v = 2 * inputs.splitmix_uniform(9, 0, 12, 10) - 1
    assert abs((g * v).sum() / _fd(c, rho0, sf, "rho", 1e-5, v) - 1) < 1e-6
    for (y, x) in ((0, 0), (5, 6), (9, 11)):
        e = np.zeros_like(rho0)
        e[y, x] = 1.0
        fd = _fd(c, rho0, sf, "rho", 1e-5, e)
        assert abs(g[y, x] - fd) < 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


def test_finite_differences_catch_a_planted_adjoint_mistake():
    """An adjoint that ignores the correction term C (forward unchanged)
    disagrees with the finite differences."""
    c, rho0, sf = _setup(O.IMPROVED, O.BGK, flags=O.FLAG_ADJOINT_DROP_C)
    _, g, gk, _ = O.adjoint(c, rho0, N, U_FROM, sf)
    c_ok = dataclasses.replace(c, flags=0)
    assert abs(gk / _fd(c_ok, rho0, sf, "kappa", 1e-6) - 1) > 1e-4
