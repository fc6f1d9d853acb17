"""Thin Python binding of liblbfe (the C ABI in include/lbfe.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of liblbfe. PyTorch supplies the device workspace and the CUDA stream. The
library must have been built (``paper_2008_01473_gb300.build.build()``); if it
is missing, importing the binding's loader raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields as dc_fields

import numpy as np

from .build import LIB

STANDARD, IMPROVED, STANDARD_PT = 0, 1, 2  # STANDARD_PT: Eq. 13 left (pressure-tensor force)
IMPROVED_SMOOTH = 3  # improved scheme, Eq. 29 on the lattice-weight average of phi u
LAX_WENDROFF = 4  # the comparison scheme of Appendix A (Eqs. A1-A4)
BGK, MRT = 0, 1
VDW, CS = 0, 1
FP64, FP32 = 0, 1

_STATUS = {0: "LB_OK", 1: "LB_E_INVALID", 2: "LB_E_CUDA", 3: "LB_E_UNSTABLE", 4: "LB_E_TIMEOUT",
           5: "LB_E_WORKSPACE", 6: "LB_E_STATE"}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _CWindow(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("c", C.c_double), ("d", C.c_double)]


WIN_RECT, WIN_DISC = 0, 1


class _CCase(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("scheme", C.c_int32), ("collision", C.c_int32),
                ("eos", C.c_int32), ("walls", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("R", C.c_double), ("T", C.c_double), ("kappa", C.c_double), ("tau_v", C.c_double),
                ("tau_e", C.c_double), ("tau_s", C.c_double), ("tau_q", C.c_double),
                ("pm_c0", C.c_double), ("nu", C.c_double), ("rho_ref", C.c_double), ("wall_u", C.c_double),
                ("rho_wall", C.c_double), ("lw_A", C.c_double), ("lw_B", C.c_double)]


@dataclass
class Case:
    """One periodic case (mirrors ``lb_case``)."""
    nx: int
    ny: int
    scheme: int = IMPROVED
    collision: int = BGK
    eos: int = VDW
    a: float = 9.0 / 392.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    T: float = 0.8 / 14.0
    kappa: float = 0.02
    tau_v: float = 1.0
    tau_e: float = 1.0
    tau_s: float = 1.0
    tau_q: float = 1.1
    pm_c0: float = 1.0
    nu: float = 0.0
    rho_ref: float = 0.0
    walls: int = 0          # 1: moving no-slip walls below y = 0 and above y = ny - 1
    wall_u: float = 0.0     # x velocity of both walls
    rho_wall: float = 0.0   # density of the wall state (> 0 with walls)
    lw_A: float = 0.0       # LAX_WENDROFF: CFL number A, the time step (Appendix A)
    lw_B: float = 0.0       # LAX_WENDROFF: B of Eq. A3 (nu = c_s^2 (tau - 1/2 - B) A)

    def cstruct(self) -> _CCase:
        kw = {f.name: getattr(self, f.name) for f in dc_fields(self)}
        return _CCase(**kw)


_lib = None


def lib() -> C.CDLL:
    """Load liblbfe; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"liblbfe is not built ({LIB} missing); run paper_2008_01473_gb300.build.build()")
        L = C.CDLL(LIB)
        vp, i32, i64, dp, sz = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_size_t
        cp = C.POINTER(_CCase)
        L.lb_workspace_bytes.argtypes = [cp, i32, i32, C.POINTER(sz)]
        L.lb_create.argtypes = [cp, i32, i32, vp, sz, vp, C.POINTER(vp)]
        L.lb_init_fields.argtypes = [vp, i32, vp, vp, vp, i32]
        L.lb_init_fields_f32.argtypes = [vp, i32, vp, vp, vp, i32]
        L.lb_moments_f32.argtypes = [vp, i32, vp, vp, vp, vp, i32]
        L.lb_step.argtypes = [vp, i64]
        L.lb_moments.argtypes = [vp, i32, vp, vp, vp, vp, i32]
        L.lb_reductions.argtypes = [vp, dp, C.POINTER(i32)]
        L.lb_snapshot_bytes.argtypes = [vp, i32, C.POINTER(sz)]
        L.lb_save.argtypes = [vp, i32, vp, sz]
        L.lb_load.argtypes = [vp, i32, vp, sz]
        L.lb_critical.argtypes = [i32, C.c_double, C.c_double, C.c_double, dp, dp]
        L.lb_maxwell.argtypes = [i32, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
        L.lb_surface_tension.argtypes = [i32] + [C.c_double] * 5 + [dp]
        L.lb_young_laplace.argtypes = [i32] + [C.c_double] * 6 + [dp, dp]
        L.lb_fields_static.argtypes = [cp, i32, vp, C.c_double, vp, vp, vp, vp, vp, vp]
        L.lb_adjoint_workspace_bytes.argtypes = [vp, i32, i64, i32, C.POINTER(sz)]
        L.lb_adjoint_step.argtypes = [vp, i32, vp, i64, i64, vp, i32, i32, vp, sz, dp, vp, dp, dp]
        L.lb_worklist.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
        L.lb_wait_selftest.argtypes = [vp]
        L.lb_launch_mode.argtypes = [vp, i32, C.POINTER(i32)]
        L.lb_persistent_selftest.argtypes = [vp, i64]
        L.lb_window_means.argtypes = [vp, i32, i32, C.POINTER(_CWindow), dp]
        L.lb_step_stats_bytes.argtypes = [vp, i32, C.POINTER(sz)]
        L.lb_step_stats_attach.argtypes = [vp, vp, sz, i32]
        L.lb_step_stats_range.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i64)]
        L.lb_step_stats_read.argtypes = [vp, i32, i64, i32, dp]
        L.lb_last_error.argtypes = [vp]
        L.lb_last_error.restype = C.c_char_p
        L.lb_destroy.argtypes = [vp]
        L.lb_destroy.restype = None
        for name in ("lb_workspace_bytes", "lb_create", "lb_init_fields", "lb_init_fields_f32", "lb_step",
                     "lb_moments", "lb_moments_f32",
                     "lb_reductions", "lb_snapshot_bytes", "lb_save", "lb_load", "lb_critical", "lb_maxwell",
                     "lb_fields_static", "lb_adjoint_workspace_bytes", "lb_adjoint_step", "lb_worklist",
                     "lb_wait_selftest", "lb_window_means", "lb_launch_mode", "lb_persistent_selftest",
                     "lb_surface_tension", "lb_young_laplace", "lb_step_stats_bytes", "lb_step_stats_attach",
                     "lb_step_stats_range", "lb_step_stats_read"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st: int, h=None, what: str = ""):
    if st != 0:
        msg = lib().lb_last_error(h).decode() if h else what
        raise LBError(st, msg or what)


def critical(eos: int, a: float, b: float, R: float = 1.0) -> tuple[float, float]:
    """(T_c, rho_c) from the host solver of liblbfe."""
    tc, rc = C.c_double(), C.c_double()
    _check(lib().lb_critical(eos, a, b, R, C.byref(tc), C.byref(rc)), what="lb_critical")
    return tc.value, rc.value


def surface_tension(eos: int, a: float, b: float, R: float, T: float, kappa: float) -> float:
    """Flat-interface square-gradient tension at coexistence (host solver)."""
    out = C.c_double()
    _check(lib().lb_surface_tension(eos, a, b, R, T, kappa, C.byref(out)), what="lb_surface_tension")
    return out.value


def young_laplace(eos: int, a: float, b: float, R: float, T: float, sigma: float, r: float) -> tuple[float, float]:
    """(rho_g, rho_l) around a droplet of radius r by Eq. 32 (host solver)."""
    g, l = C.c_double(), C.c_double()
    _check(lib().lb_young_laplace(eos, a, b, R, T, sigma, r, C.byref(g), C.byref(l)), what="lb_young_laplace")
    return g.value, l.value


def maxwell(eos: int, a: float, b: float, R: float, T: float) -> tuple[float, float]:
    """Maxwell coexistence densities (rho_g, rho_l) from the host solver of liblbfe."""
    g, l = C.c_double(), C.c_double()
    _check(lib().lb_maxwell(eos, a, b, R, T, C.byref(g), C.byref(l)), what="lb_maxwell")
    return g.value, l.value


def _host_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Lattice:
    """A set of independent periodic cases stepped together on one GPU."""

    def __init__(self, cases, precision: int = FP32, device=None, stream=None):
        import torch

        self.cases = list(cases)
        self.precision = precision
        self._torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        arr = (_CCase * len(self.cases))(*[c.cstruct() for c in self.cases])
        self._carr = arr
        nb = C.c_size_t()
        _check(lib().lb_workspace_bytes(arr, len(self.cases), precision, C.byref(nb)),
               what="lb_workspace_bytes: invalid case parameters")
        self.workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(lib().lb_create(arr, len(self.cases), precision, C.c_void_p(self._ws_ptr), nb.value,
                               C.c_void_p(self.stream.cuda_stream), C.byref(h)), what="lb_create")
        self._h = h

    # ------------------------------------------------------------------ helpers
    def _ptr_of(self, a, shape, fp32: bool = False):
        """(pointer, on_device, keepalive) for a host array or a CUDA tensor of
        FP64 (FP32 with fp32)."""
        torch = self._torch
        if a is None:
            return None, 0, None
        if isinstance(a, torch.Tensor) and a.is_cuda:
            t = a.detach().to(torch.float32 if fp32 else torch.float64).contiguous()
            assert tuple(t.shape) == shape, (t.shape, shape)
            return C.c_void_p(t.data_ptr()), 1, t
        h = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
        h = np.ascontiguousarray(np.asarray(h, dtype=np.float32)) if fp32 else _host_f64(h)
        assert h.shape == shape, (h.shape, shape)
        return C.c_void_p(h.ctypes.data), 0, h

    def _shape(self, case_id):
        c = self.cases[case_id]
        return (c.ny, c.nx)

    # ---------------------------------------------------------------------- API
    def init_fields(self, case_id: int, rho0, ux0=None, uy0=None, fp32: bool = False):
        """Initial state of case_id from rho0 (and u0): FP64 fields, or FP32
        ones with fp32 (lb_init_fields_f32)."""
        sh = self._shape(case_id)
        p, dev, k0 = self._ptr_of(rho0, sh, fp32)
        pu, devu, k1 = self._ptr_of(ux0, sh, fp32)
        pv, devv, k2 = self._ptr_of(uy0, sh, fp32)
        if (ux0 is not None and devu != dev) or (uy0 is not None and devv != dev):
            raise ValueError("rho0, ux0 and uy0 must all be on the host or all on the device")
        fn = lib().lb_init_fields_f32 if fp32 else lib().lb_init_fields
        _check(fn(self._h, case_id, p, pu, pv, dev), self._h)
        del k0, k1, k2

    def step(self, nsteps: int = 1):
        _check(lib().lb_step(self._h, int(nsteps)), self._h)

    def window_means(self, case_id: int, windows):
        """Mean of rho over each window, summed on the GPU in FP64: windows
        are ("rect", x0, y0, w, h) (periodic) or ("disc", cx, cy, r)."""
        arr = (_CWindow * max(1, len(windows)))()
        for k, w in enumerate(windows):
            if w[0] == "rect":
                arr[k] = _CWindow(WIN_RECT, 0, float(w[1]), float(w[2]), float(w[3]), float(w[4]))
            elif w[0] == "disc":
                arr[k] = _CWindow(WIN_DISC, 0, float(w[1]), float(w[2]), float(w[3]), 0.0)
            else:
                raise ValueError(f"unknown window {w[0]!r}")
        out = np.empty(max(1, len(windows)))
        _check(lib().lb_window_means(self._h, case_id, len(windows), arr,
                                     out.ctypes.data_as(C.POINTER(C.c_double))), self._h)
        return out[:len(windows)]

    def wait_selftest(self):
        """Enqueue the failure-detection self-test (a bounded wait that gives
        up); the next reductions() call reports LB_E_TIMEOUT."""
        _check(lib().lb_wait_selftest(self._h), self._h)

    def launch_mode(self, mode: int = -1) -> bool:
        """Set the persistent-launch mode (0 never, 1 always, 2 automatic;
        -1 keeps it) and return whether the persistent launch is in use."""
        p = C.c_int32()
        _check(lib().lb_launch_mode(self._h, int(mode), C.byref(p)), self._h)
        return bool(p.value)

    def persistent_selftest(self, nsteps: int = 8):
        """Enqueue the persistent launch's failure-detection self-test (a
        wait that nothing completes gives up); the next reductions() call
        reports LB_E_TIMEOUT."""
        _check(lib().lb_persistent_selftest(self._h, int(nsteps)), self._h)

    def worklist(self):
        """(rows per segment, item count, narrow blocks used) of the work-list
        in use; 0 rows is the slot-share rule."""
        r, n, w = C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().lb_worklist(self._h, C.byref(r), C.byref(n), C.byref(w)), self._h)
        return r.value, n.value, bool(w.value)

    def moments(self, case_id: int, on_device: bool = False, fp32: bool = False):
        """dict rho, ux, uy, mu of the current state (numpy, or CUDA tensors);
        FP64, or FP32 with fp32 (lb_moments_f32)."""
        sh = self._shape(case_id)
        torch = self._torch
        if on_device:
            dt = torch.float32 if fp32 else torch.float64
            out = {k: torch.empty(sh, dtype=dt, device=self.device) for k in ("rho", "ux", "uy", "mu")}
            ptrs = [C.c_void_p(out[k].data_ptr()) for k in ("rho", "ux", "uy", "mu")]
        else:
            out = {k: np.empty(sh, dtype=np.float32 if fp32 else np.float64) for k in ("rho", "ux", "uy", "mu")}
            ptrs = [C.c_void_p(out[k].ctypes.data) for k in ("rho", "ux", "uy", "mu")]
        fn = lib().lb_moments_f32 if fp32 else lib().lb_moments
        _check(fn(self._h, case_id, *ptrs, 1 if on_device else 0), self._h)
        return out

    def reductions(self, raise_unstable: bool = False):
        """(out[ncases, 5] = mass, ke, umax, steps, 0; status[ncases])."""
        n = len(self.cases)
        out = np.zeros((n, 5))
        st = np.zeros(n, dtype=np.int32)
        rc = lib().lb_reductions(self._h, out.ctypes.data_as(C.POINTER(C.c_double)),
                                 st.ctypes.data_as(C.POINTER(C.c_int32)))
        if rc != 0 and (rc != 3 or raise_unstable):
            _check(rc, self._h)
        return out, st

    def attach_step_stats(self, history: int = 1024):
        """Record per-step statistics of every case (mass, kinetic energy,
        max |u|, node count of the state each step starts from) in a device
        ring of `history` entries per case; history 0 detaches."""
        if history <= 0:
            _check(lib().lb_step_stats_attach(self._h, None, 0, 0), self._h)
            self._stats_buf = None
            return
        nb = C.c_size_t()
        _check(lib().lb_step_stats_bytes(self._h, int(history), C.byref(nb)), self._h, "lb_step_stats_bytes")
        buf = self._torch.empty(nb.value + 256, dtype=self._torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        _check(lib().lb_step_stats_attach(self._h, C.c_void_p(ptr), nb.value, int(history)), self._h)
        self._stats_buf = buf  # the library does not own it

    def step_stats(self, case_id: int, first=None, count=None):
        """(first state, array[count, 4] of mass, kinetic energy, max |u|,
        nodes) of the recorded states of case_id (all those still held by
        default)."""
        f, n = C.c_int64(), C.c_int64()
        _check(lib().lb_step_stats_range(self._h, case_id, C.byref(f), C.byref(n)), self._h)
        first = f.value if first is None else int(first)
        count = f.value + n.value - first if count is None else int(count)
        out = np.zeros((max(count, 0), 4))
        _check(lib().lb_step_stats_read(self._h, case_id, first, count, out.ctypes.data_as(C.POINTER(C.c_double))),
               self._h)
        return first, out

    def adjoint(self, case_id: int, rho0, nsteps: int, u_from: int, s_final=None, ckpt_every: int = 0):
        """Loss L = sum_{n >= u_from} sum |u^n|^2 + sum s_final rho^N of a run from
        rho0, and (L, dL/drho0, dL/dkappa, dL/dT) by the library's adjoint
        (FP64 handles in FP64, FP32 handles in FP32). Arrays on the host or CUDA
        tensors (results follow rho0)."""
        torch = self._torch
        sh = self._shape(case_id)
        nb = C.c_size_t()
        _check(lib().lb_adjoint_workspace_bytes(self._h, case_id, int(nsteps), int(ckpt_every), C.byref(nb)),
               self._h, "lb_adjoint_workspace_bytes")
        ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        wsp = (ws.data_ptr() + 255) // 256 * 256
        p, dev, k0 = self._ptr_of(rho0, sh)
        ps, devs, k1 = self._ptr_of(s_final, sh)
        if s_final is not None and devs != dev:
            raise ValueError("rho0 and s_final must both be on the host or both on the device")
        if dev:
            grad = torch.empty(sh, dtype=torch.float64, device=self.device)
            gp = C.c_void_p(grad.data_ptr())
        else:
            grad = np.empty(sh)
            gp = C.c_void_p(grad.ctypes.data)
        L, gk, gT = C.c_double(), C.c_double(), C.c_double()
        _check(lib().lb_adjoint_step(self._h, case_id, p, int(nsteps), int(u_from), ps, dev, int(ckpt_every),
                                C.c_void_p(wsp), nb.value, C.byref(L), gp, C.byref(gk), C.byref(gT)), self._h)
        del k0, k1, ws
        return L.value, grad, gk.value, gT.value

    def save(self, case_id: int) -> bytes:
        nb = C.c_size_t()
        _check(lib().lb_snapshot_bytes(self._h, case_id, C.byref(nb)), self._h)
        buf = (C.c_uint8 * nb.value)()
        _check(lib().lb_save(self._h, case_id, buf, nb.value), self._h)
        return bytes(buf)

    def load(self, case_id: int, snap: bytes):
        buf = (C.c_uint8 * len(snap)).from_buffer_copy(snap)
        _check(lib().lb_load(self._h, case_id, buf, len(snap)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
