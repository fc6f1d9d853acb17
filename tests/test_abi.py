"""CPU-side checks of the C ABI: the library builds and loads, it exports every
function include/lbfe.h declares, parameter validation works without a GPU,
and the host thermodynamics agree with the oracle's independent solver."""
import ctypes as C
import os
import re

import pytest

import oracle as O
from oracle import thermo
from paper_2008_01473_gb300 import build as B
from paper_2008_01473_gb300 import lbfe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbfe.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_validation(lib):
    ok = lbfe.Case(nx=64, ny=48)
    nb = C.c_size_t()
    arr = (lbfe._CCase * 1)(ok.cstruct())
    assert lib.lb_workspace_bytes(arr, 1, lbfe.FP32, C.byref(nb)) == 0
    n32 = nb.value
    assert lib.lb_workspace_bytes(arr, 1, lbfe.FP64, C.byref(nb)) == 0
    assert nb.value > n32 > 2 * 9 * 64 * 48 * 4
    c3 = lbfe.Case(**{**ok.__dict__, "scheme": lbfe.IMPROVED_SMOOTH})
    assert lib.lb_workspace_bytes((lbfe._CCase * 1)(c3.cstruct()), 1, lbfe.FP32, C.byref(nb)) == 0
    lw = dict(scheme=lbfe.LAX_WENDROFF, collision=lbfe.BGK, lw_A=0.1, lw_B=-0.7)
    c4 = lbfe.Case(**{**ok.__dict__, **lw})
    assert lib.lb_workspace_bytes((lbfe._CCase * 1)(c4.cstruct()), 1, lbfe.FP64, C.byref(nb)) == 0
    for bad in (dict(nx=2), dict(tau_v=0.5), dict(kappa=0.0), dict(scheme=5), dict(T=float("nan")),
                dict(nu=-1.0), {**lw, "lw_A": 0.0}, {**lw, "lw_A": 1.5}, {**lw, "collision": lbfe.MRT},
                {**lw, "lw_B": 0.5}, {**lw, "nu": 0.1}, {**lw, "walls": 1, "rho_wall": 1.0}):
        c = lbfe.Case(**{**ok.__dict__, **bad})
        arr = (lbfe._CCase * 1)(c.cstruct())
        assert lib.lb_workspace_bytes(arr, 1, lbfe.FP32, C.byref(nb)) == 1, bad
    assert lib.lb_workspace_bytes(arr, 0, lbfe.FP32, C.byref(nb)) == 1
    # largest lattice: 9 ny pitch elements must stay below 2^31 (32-bit offsets)
    for ny, st in ((14563, 0), (14564, 1)):
        c = lbfe.Case(**{**ok.__dict__, "nx": 16384, "ny": ny})
        arr = (lbfe._CCase * 1)(c.cstruct())
        assert lib.lb_workspace_bytes(arr, 1, lbfe.FP32, C.byref(nb)) == st, ny
    h = C.c_void_p()
    arr = (lbfe._CCase * 1)(ok.cstruct())
    # misaligned / too small workspace is rejected before any device call
    assert lib.lb_create(arr, 1, lbfe.FP32, C.c_void_p(8), 16, None, C.byref(h)) == 5


@pytest.mark.parametrize("t", [0.95, 0.9, 0.8, 0.7, 0.6, 0.5])
@pytest.mark.parametrize("eos", ["vdw", "cs"])
def test_host_maxwell_matches_oracle(lib, eos, t):
    e = thermo.vdw_paper() if eos == "vdw" else thermo.EOS(thermo.CS, 9 / 392, 9 / 98)
    tc, rc = lbfe.critical(e.kind, e.a, e.b, e.R)
    tc_o, rc_o = e.critical()
    assert abs(tc / tc_o - 1) < 1e-12 and abs(rc / rc_o - 1) < 1e-6
    T, rg_o, rl_o = thermo.maxwell_reduced(e, t)
    rg, rl = lbfe.maxwell(e.kind, e.a, e.b, e.R, T)
    assert abs(rg / rg_o - 1) < 1e-11 and abs(rl / rl_o - 1) < 1e-12


@pytest.mark.parametrize("t", [0.9, 0.8, 0.7])
@pytest.mark.parametrize("eos", ["vdw", "cs"])
def test_host_tension_and_young_laplace_match_oracle(lib, eos, t):
    """The library's surface tension (Gauss-Legendre) and Eq. 32 densities
    against the oracle's (adaptive quadrature, brentq)."""
    e = thermo.vdw_paper() if eos == "vdw" else thermo.EOS(thermo.CS, 9 / 392, 9 / 98)
    T, _, _ = thermo.maxwell_reduced(e, t)
    sig = lbfe.surface_tension(e.kind, e.a, e.b, e.R, T, 0.02)
    sig_o = e.surface_tension(T, 0.02)
    assert abs(sig / sig_o - 1) < 1e-9
    for r in (12.0, 25.0, 40.0):
        g, l = lbfe.young_laplace(e.kind, e.a, e.b, e.R, T, sig, r)
        g_o, l_o = e.young_laplace(T, sig_o, r)
        assert abs(g / g_o - 1) < 1e-9 and abs(l / l_o - 1) < 1e-9


def test_host_maxwell_rejects_supercritical(lib):
    e = thermo.vdw_paper()
    with pytest.raises(lbfe.LBError):
        lbfe.maxwell(e.kind, e.a, e.b, e.R, 1.01 / 14)
