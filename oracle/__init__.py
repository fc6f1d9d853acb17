"""Python face of the FP64 CPU oracle (``lbfe_oracle.c``) and its thermodynamics.

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the product library never does, and
nothing here imports the product library.

``build()`` compiles ``lbfe_oracle.c`` with gcc into ``oracle/_build`` (plain
C, ``-O2 -ffp-contract=off`` so that the literal expressions round as
written). Arrays cross the boundary as C-contiguous float64 numpy arrays:
populations ``f[9, ny, nx]`` and fields ``[ny, nx]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

from . import thermo

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbfe_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblbfe_oracle.so")
_lib = None

STANDARD, IMPROVED, STANDARD_PT = 0, 1, 2  # STANDARD_PT: Eq. 13 left (pressure-tensor force)
IMPROVED_SMOOTH = 3  # improved scheme, Eq. 29's derivatives of the lattice-weight average of phi u
LAX_WENDROFF = 4  # the comparison scheme of Appendix A (Eqs. A1-A4): BGK, standard force, dt = A
BGK, MRT = 0, 1
VDW, CS = thermo.VDW, thermo.CS

# planted-mistake hooks (pin tests only)
FLAG_DROP_C = 1
FLAG_FLIP_HALF_FORCE = 2
FLAG_ADJOINT_DROP_C = 4
FLAG_WALL_EVEN_JY = 8
FLAG_NU_SWAPPED = 16
FLAG_NU_STANDARD_MAP = 32
FLAG_MEQ_DROP_U2 = 64  # the standard e-equilibrium without its rho |u|^2 term


class _CCase(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("scheme", C.c_int32),
                ("collision", C.c_int32), ("eos", C.c_int32), ("flags", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T", C.c_double),
                ("kappa", C.c_double), ("tau_v", C.c_double), ("tau_e", C.c_double),
                ("tau_s", C.c_double), ("tau_q", C.c_double), ("pm_c0", C.c_double),
                ("nu", C.c_double), ("walls", C.c_int32), ("pad_", C.c_int32), ("wall_u", C.c_double),
                ("rho_wall", C.c_double), ("lw_A", C.c_double), ("lw_B", C.c_double)]


@dataclass
class Case:
    """One periodic lattice and its parameters (mirrors ``orc_case``)."""
    nx: int
    ny: int
    scheme: int = IMPROVED
    collision: int = BGK
    eos: int = CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    kappa: float = 0.02
    tau_v: float = 1.0
    tau_e: float = 1.0
    tau_s: float = 1.0
    tau_q: float = 1.1
    pm_c0: float = 1.0
    nu: float = 0.0
    flags: int = 0
    walls: int = 0          # 1: moving no-slip walls below y = 0 and above y = ny - 1
    wall_u: float = 0.0     # x velocity of both walls
    rho_wall: float = 0.0   # density in the moving-wall term
    lw_A: float = 0.0       # LAX_WENDROFF: CFL number A (the time step, Appendix A)
    lw_B: float = 0.0       # LAX_WENDROFF: B of Eq. A3 (nu = c_s^2 (tau - 1/2 - B) A)
    _c: _CCase = field(default=None, repr=False, compare=False)

    def cstruct(self) -> _CCase:
        return _CCase(self.nx, self.ny, self.scheme, self.collision, self.eos, self.flags,
                      self.a, self.b, self.R, self.T, self.kappa, self.tau_v, self.tau_e,
                      self.tau_s, self.tau_q, self.pm_c0, self.nu, self.walls, 0, self.wall_u,
                      self.rho_wall, self.lw_A, self.lw_B)

    def thermo(self) -> thermo.EOS:
        return thermo.EOS(self.eos, self.a, self.b, self.R)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C) if it is missing or stale."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i32, i64 = C.c_double, C.c_int32, C.c_int64
        dp = P(d)
        cp = P(_CCase)
        _lib.orc_Ef.argtypes = [cp, d]; _lib.orc_Ef.restype = d
        _lib.orc_dEf.argtypes = [cp, d]; _lib.orc_dEf.restype = d
        _lib.orc_pEOS.argtypes = [cp, d]; _lib.orc_pEOS.restype = d
        _lib.orc_grad.argtypes = [C.c_int, C.c_int, dp, dp, dp]; _lib.orc_grad.restype = None
        _lib.orc_laplacian.argtypes = [C.c_int, C.c_int, dp, dp]; _lib.orc_laplacian.restype = None
        _lib.orc_M.argtypes = [dp]; _lib.orc_M.restype = None
        _lib.orc_Minv.argtypes = [dp]; _lib.orc_Minv.restype = None
        _lib.orc_meq.argtypes = [cp, d, d, d, d, dp]; _lib.orc_meq.restype = None
        _lib.orc_feq.argtypes = [cp, d, d, d, d, dp]; _lib.orc_feq.restype = None
        _lib.orc_guo.argtypes = [d, d, d, d, dp]; _lib.orc_guo.restype = None
        _lib.orc_fields.argtypes = [cp, dp] + [dp] * 8; _lib.orc_fields.restype = C.c_int
        _lib.orc_step.argtypes = [cp, dp, i64]; _lib.orc_step.restype = i64
        _lib.orc_init.argtypes = [cp, dp, dp, dp, dp]; _lib.orc_init.restype = C.c_int
        _lib.orc_adjoint.argtypes = [cp, dp, i64, i64, dp, dp, dp, dp, dp]; _lib.orc_adjoint.restype = C.c_int
        del i32
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- thermo
def dEf(case: Case, rho: float) -> float:
    return lib().orc_dEf(C.byref(case.cstruct()), float(rho))


def pEOS(case: Case, rho: float) -> float:
    return lib().orc_pEOS(C.byref(case.cstruct()), float(rho))


def Ef(case: Case, rho: float) -> float:
    return lib().orc_Ef(C.byref(case.cstruct()), float(rho))


# -------------------------------------------------------------- stencils
def grad(phi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 17 isotropic gradient on a periodic lattice ``phi[ny, nx]``."""
    phi = _f64(phi)
    ny, nx = phi.shape
    gx, gy = np.empty_like(phi), np.empty_like(phi)
    lib().orc_grad(nx, ny, _ptr(phi), _ptr(gx), _ptr(gy))
    return gx, gy


def laplacian(phi: np.ndarray) -> np.ndarray:
    phi = _f64(phi)
    ny, nx = phi.shape
    out = np.empty_like(phi)
    lib().orc_laplacian(nx, ny, _ptr(phi), _ptr(out))
    return out


# -------------------------------------------------------- moment algebra
def M() -> np.ndarray:
    out = np.empty(81)
    lib().orc_M(_ptr(out))
    return out.reshape(9, 9)


def Minv() -> np.ndarray:
    out = np.empty(81)
    lib().orc_Minv(_ptr(out))
    return out.reshape(9, 9)


def meq(case: Case, rho: float, ux: float, uy: float, mu: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_meq(C.byref(case.cstruct()), rho, ux, uy, mu, _ptr(out))
    return out


def feq(case: Case, rho: float, ux: float, uy: float, mu: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_feq(C.byref(case.cstruct()), rho, ux, uy, mu, _ptr(out))
    return out


def guo(ux: float, uy: float, Fx: float, Fy: float) -> np.ndarray:
    out = np.empty(9)
    lib().orc_guo(ux, uy, Fx, Fy, _ptr(out))
    return out


# --------------------------------------------------------------- lattice
def init(case: Case, rho0: np.ndarray, ux0=None, uy0=None) -> np.ndarray:
    """f(0) = M^-1 m_eq(rho0, u0) of the case's scheme; returns f[9, ny, nx]."""
    rho0 = _f64(rho0)
    assert rho0.shape == (case.ny, case.nx)
    ux0 = None if ux0 is None else _f64(ux0)
    uy0 = None if uy0 is None else _f64(uy0)
    f = np.empty((9, case.ny, case.nx))
    rc = lib().orc_init(C.byref(case.cstruct()), _ptr(rho0), _ptr(ux0), _ptr(uy0), _ptr(f))
    if rc != 0:
        raise ValueError("initial density must be positive")
    return f


def step(case: Case, f: np.ndarray, nsteps: int) -> int:
    """Advance ``f`` in place; returns the number of steps completed."""
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (9, case.ny, case.nx)
    return int(lib().orc_step(C.byref(case.cstruct()), _ptr(f), int(nsteps)))


@dataclass
class Fields:
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    mu: np.ndarray
    Fx: np.ndarray
    Fy: np.ndarray
    C1: np.ndarray
    C7: np.ndarray
    ok: bool


def fields(case: Case, f: np.ndarray) -> Fields:
    """Macroscopic fields of the state ``f`` (stages 1-7 of a step)."""
    f = _f64(f)
    sh = (case.ny, case.nx)
    arrs = [np.empty(sh) for _ in range(8)]
    rc = lib().orc_fields(C.byref(case.cstruct()), _ptr(f), *[_ptr(a) for a in arrs])
    return Fields(*arrs, ok=(rc == 0))


def reductions(case: Case, f: np.ndarray) -> dict:
    """Mass, kinetic energy sum(rho |u|^2 / 2) and max |u| (FP64)."""
    fl = fields(case, f)
    u2 = fl.ux**2 + fl.uy**2
    return {"mass": float(fl.rho.sum()), "ke": float(0.5 * (fl.rho * u2).sum()),
            "umax": float(np.sqrt(u2.max()))}


def adjoint(case: Case, rho0: np.ndarray, nsteps: int, u_from: int, s_final=None):
    """Loss L = sum_{n=u_from}^{nsteps} sum_x |u^n|^2 + sum_x s_final rho^N and its
    gradients (dL/drho0, dL/dkappa, dL/dT) by the oracle's reverse sweep."""
    rho0 = _f64(rho0)
    assert rho0.shape == (case.ny, case.nx)
    sf = None if s_final is None else _f64(s_final)
    g = np.empty_like(rho0)
    L, gk, gT = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_adjoint(C.byref(case.cstruct()), _ptr(rho0), int(nsteps), int(u_from), _ptr(sf), C.byref(L),
                           _ptr(g), C.byref(gk), C.byref(gT))
    if rc != 0:
        raise ValueError("oracle adjoint failed (non-physical state or nu > 0)")
    return L.value, g, gk.value, gT.value


def loss(case: Case, rho0: np.ndarray, nsteps: int, u_from: int, s_final=None) -> float:
    """The loss of adjoint() from a plain forward run."""
    f = init(case, rho0)
    L = 0.0
    for n in range(nsteps + 1):
        if n >= u_from or n == nsteps:
            fl = fields(case, f)
            if n >= u_from:
                L += float((fl.ux ** 2 + fl.uy ** 2).sum())
            if n == nsteps and s_final is not None:
                L += float((np.asarray(s_final) * fl.rho).sum())
        if n < nsteps:
            assert step(case, f, 1) == 1
    return L
