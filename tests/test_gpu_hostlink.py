"""Host buffers of lb_init_fields and lb_moments: page-locked host memory is
read and written by the kernels themselves over the host link, pageable
memory is staged through the workspace; both give the same bits as device
buffers."""
import ctypes as C

import numpy as np
import pytest

from oracle import thermo
from paper_2008_01473_gb300 import inputs, lbfe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_01473_gb300 import build

    build.build()


def _pops(lat, nx, ny):
    """Snapshot header and the stored populations at the lattice columns (the
    row padding up to the pitch is never written)."""
    snap = lat.save(0)
    dt = np.float32 if lat.precision == lbfe.FP32 else np.float64
    pitch = (nx + 31) // 32 * 32
    raw = np.frombuffer(snap[16:], dtype=dt).reshape(9, ny, pitch)[:, :, :nx]
    return np.concatenate([np.frombuffer(snap[:16], dtype=np.uint8).astype(np.float64),
                           raw.astype(np.float64).ravel()])


@pytest.mark.parametrize("precision", [lbfe.FP32, lbfe.FP64])
@pytest.mark.parametrize("shape", [(96, 72), (37, 29)])
def test_pinned_host_buffers_match_pageable_and_device(precision, shape):
    import torch

    nx, ny = shape
    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, 0.8)
    case = lbfe.Case(nx=nx, ny=ny, scheme=lbfe.IMPROVED, collision=lbfe.MRT, eos=lbfe.VDW, a=e.a, b=e.b, R=1.0,
                     T=T, kappa=0.02, tau_v=0.8)
    rho0 = inputs.droplet(nx, ny, 0.3 * min(nx, ny), rl, rg, width=3.0, noise=1e-3, seed=9)
    pinned = torch.from_numpy(rho0.copy()).pin_memory()
    a = lbfe.Lattice([case], precision=precision)
    b = lbfe.Lattice([case], precision=precision)
    a.init_fields(0, rho0)     # pageable: staged
    b.init_fields(0, pinned)   # page-locked: read by the init kernel
    assert np.array_equal(_pops(a, nx, ny), _pops(b, nx, ny))
    a.step(7)
    names = ("rho", "ux", "uy", "mu")
    pin_out = {k: torch.empty((ny, nx), dtype=torch.float64).pin_memory() for k in names}
    lbfe._check(lbfe.lib().lb_moments(a._h, 0, *[C.c_void_p(pin_out[k].data_ptr()) for k in names], 0), a._h)
    host = a.moments(0)                    # pageable outputs
    dev = a.moments(0, on_device=True)     # device outputs
    for k in names:
        assert np.array_equal(pin_out[k].numpy(), host[k]), k
        assert np.array_equal(dev[k].cpu().numpy(), host[k]), k
    # a subset of outputs (the others NULL), mixed page-locked and pageable
    rho_only = torch.zeros((ny, nx), dtype=torch.float64).pin_memory()
    uy_host = np.zeros((ny, nx))
    lbfe._check(lbfe.lib().lb_moments(a._h, 0, C.c_void_p(rho_only.data_ptr()), None,
                                      C.c_void_p(uy_host.ctypes.data), None, 0), a._h)
    assert np.array_equal(rho_only.numpy(), host["rho"]) and np.array_equal(uy_host, host["uy"])
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [lbfe.FP32, lbfe.FP64])
def test_fp32_field_calls(precision):
    """lb_init_fields_f32 gives the state lb_init_fields gives from the same
    values widened to FP64 (pageable, page-locked and device inputs, with
    FP32 initial velocities), and lb_moments_f32 returns lb_moments' values
    rounded to FP32 (pageable, page-locked and device outputs)."""
    import torch

    nx, ny = 68, 37
    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, 0.8)
    case = lbfe.Case(nx=nx, ny=ny, scheme=lbfe.IMPROVED, collision=lbfe.MRT, eos=lbfe.VDW, a=e.a, b=e.b, R=1.0,
                     T=T, kappa=0.02, tau_v=0.8)
    rho0 = inputs.droplet(nx, ny, 0.3 * min(nx, ny), rl, rg, width=3.0, noise=1e-3, seed=4).astype(np.float32)
    ux0 = (0.01 * (2 * inputs.splitmix_uniform(2, 0, nx, ny) - 1)).astype(np.float32)
    uy0 = (0.01 * (2 * inputs.splitmix_uniform(3, 0, nx, ny) - 1)).astype(np.float32)
    ref = lbfe.Lattice([case], precision=precision)
    ref.init_fields(0, rho0.astype(np.float64), ux0.astype(np.float64), uy0.astype(np.float64))
    want = _pops(ref, nx, ny)
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in (rho0, ux0, uy0)]
    device = [torch.from_numpy(a.copy()).cuda() for a in (rho0, ux0, uy0)]
    for src in ((rho0, ux0, uy0), pinned, device):
        lat = lbfe.Lattice([case], precision=precision)
        lat.init_fields(0, *src, fp32=True)
        assert np.array_equal(_pops(lat, nx, ny), want)
        lat.close()
    ref.step(9)
    m64 = ref.moments(0)
    names = ("rho", "ux", "uy", "mu")
    host = ref.moments(0, fp32=True)
    dev = ref.moments(0, on_device=True, fp32=True)
    pin = {k: torch.empty((ny, nx), dtype=torch.float32).pin_memory() for k in names}
    lbfe._check(lbfe.lib().lb_moments_f32(ref._h, 0, *[C.c_void_p(pin[k].data_ptr()) for k in names], 0), ref._h)
    for k in names:
        w = m64[k].astype(np.float32)
        assert host[k].dtype == np.float32 and np.array_equal(host[k], w), k
        assert np.array_equal(dev[k].cpu().numpy(), w), k
        assert np.array_equal(pin[k].numpy(), w), k
    ref.close()
