"""GPU adjoint (lb_adjoint_step) against the oracle's adjoint and against
central finite differences of the GPU's own loss (FP64 handles), the FP32
adjoint against the FP64 one, and the autograd wrapper."""
import dataclasses

import numpy as np
import pytest

import oracle as O
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


def _setup(nx, ny, scheme, collision, eos="vdw", t=0.8):
    e = thermo.vdw_paper() if eos == "vdw" else thermo.EOS(thermo.CS, 9 / 392, 9 / 98)
    T, rg, rl = thermo.maxwell_reduced(e, t)
    kw = dict(nx=nx, ny=ny, scheme=scheme, collision=collision, eos=e.kind, a=e.a, b=e.b, R=1.0, T=T,
              kappa=0.02, tau_v=0.8)
    rho0 = inputs.droplet(nx, ny, 0.3 * min(nx, ny), rl, rg, width=3.0, noise=1e-3, seed=1)
    sf = 1e-3 * (2 * inputs.splitmix_uniform(5, 0, nx, ny) - 1)
    return lbfe.Case(**kw), O.Case(**kw), rho0, sf


@pytest.mark.parametrize("scheme", [lbfe.STANDARD, lbfe.IMPROVED])
@pytest.mark.parametrize("collision", [lbfe.BGK, lbfe.MRT])
@pytest.mark.parametrize("eos", ["vdw", "cs"])
@pytest.mark.parametrize("shape,ckpt", [((12, 10), 0), ((33, 21), 7), ((257, 9), 1)])
def test_gpu_adjoint_matches_oracle(scheme, collision, eos, shape, ckpt):
    """Loss, dL/dkappa, dL/dT and dL/drho0 agree with the oracle's reverse sweep
    to 1e-10 relative (FP64 rounding order only), over checkpoint intervals
    that do and do not divide the horizon."""
    nx, ny = shape
    gc, oc, rho0, sf = _setup(nx, ny, scheme, collision, eos, t=0.9 if eos == "cs" else 0.8)
    N, uf = 27, 15
    lat = lbfe.Lattice([gc], precision=lbfe.FP64)
    L, g, gk, gT = lat.adjoint(0, rho0, N, uf, sf, ckpt)
    Lo, go, gko, gTo = O.adjoint(oc, rho0, N, uf, sf)
    assert abs(L / Lo - 1) < 1e-10
    assert abs(gk / gko - 1) < 1e-10 and abs(gT / gTo - 1) < 1e-10
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-10 * np.abs(go).max())


def test_gpu_adjoint_central_differences():
    """dL/dkappa, dL/dT and a directional dL/drho0 of the GPU adjoint equal
    central differences (FP64) of the GPU's own loss to 1e-6 relative."""
    gc, _, rho0, sf = _setup(48, 40, lbfe.IMPROVED, lbfe.MRT)
    N, uf = 120, 100

    def loss(c, r):
        lat = lbfe.Lattice([c], precision=lbfe.FP64)
        out = lat.adjoint(0, r, N, uf, sf)[0]
        lat.close()
        return out

    lat = lbfe.Lattice([gc], precision=lbfe.FP64)
    L, g, gk, gT = lat.adjoint(0, rho0, N, uf, sf, 10)
    hk, hT = 1e-6, 1e-6 * gc.T
    fdk = (loss(dataclasses.replace(gc, kappa=gc.kappa + hk), rho0) - loss(dataclasses.replace(gc, kappa=gc.kappa - hk), rho0)) / (2 * hk)
    fdT = (loss(dataclasses.replace(gc, T=gc.T + hT), rho0) - loss(dataclasses.replace(gc, T=gc.T - hT), rho0)) / (2 * hT)
    v = 2 * inputs.splitmix_uniform(3, 0, 48, 40) - 1
    fdr = (loss(gc, rho0 + 1e-5 * v) - loss(gc, rho0 - 1e-5 * v)) / 2e-5
    assert abs(gk / fdk - 1) < 1e-6
    assert abs(gT / fdT - 1) < 1e-6
    assert abs((g * v).sum() / fdr - 1) < 1e-6


def test_autograd_function():
    """LBLoss backpropagates the adjoint's gradients through torch."""
    import torch

    from paper_2008_01473_gb300.autograd import LBLoss

    gc, _, rho0, sf = _setup(24, 20, lbfe.IMPROVED, lbfe.BGK)
    kappa = torch.tensor(gc.kappa, dtype=torch.float64, requires_grad=True)
    T = torch.tensor(gc.T, dtype=torch.float64, requires_grad=True)
    r0 = torch.tensor(rho0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = LBLoss.apply(kappa, T, r0, gc, 30, 20, torch.tensor(sf, device="cuda"), 0)
    (3.0 * L).backward()
    lat = lbfe.Lattice([gc], precision=lbfe.FP64)
    Lr, g, gk, gT = lat.adjoint(0, rho0, 30, 20, sf)
    assert abs(float(L) - Lr) < 1e-12 * abs(Lr)
    assert abs(float(kappa.grad) - 3 * gk) < 1e-12 * abs(gk)
    assert abs(float(T.grad) - 3 * gT) < 1e-12 * abs(gT)
    np.testing.assert_allclose(r0.grad.cpu().numpy(), 3 * g, rtol=1e-12, atol=0)
    # no input needs a gradient: the steps alone give the same loss (no reverse sweep)
    with torch.no_grad():
        Ln = LBLoss.apply(kappa, T, r0, gc, 30, 20, torch.tensor(sf, device="cuda"), 0)
    assert abs(float(Ln) - Lr) < 1e-12 * abs(Lr)
    Ld = LBLoss.apply(kappa.detach(), T.detach(), r0.detach(), gc, 30, 0, None, 0)
    assert not Ld.requires_grad and abs(float(Ld) - lat.adjoint(0, rho0, 30, 0, None)[0]) < 1e-12 * float(Ld)
    lat.close()


@pytest.mark.parametrize("scheme", [lbfe.STANDARD, lbfe.IMPROVED])
def test_fp32_adjoint_against_fp64(scheme):
    """FP32 handles run the whole adjoint in FP32 (forward and recompute with
    the FP32 step kernel, reverse sweep in FP32; loss and parameter sums in
    FP64): loss, dL/dkappa and dL/dT within 1e-4 relative of the FP64
    adjoint, dL/drho0 within 1e-4 of its largest entry (48 x 40 droplet,
    200 steps; the differences come from the FP32 forward trajectory)."""
    gc, _, rho0, sf = _setup(48, 40, scheme, lbfe.BGK)
    r = {}
    for prec in (lbfe.FP64, lbfe.FP32):
        lat = lbfe.Lattice([gc], precision=prec)
        r[prec] = lat.adjoint(0, rho0, 200, 150, sf, 0)
        lat.close()
    (L, g, gk, gT), (L32, g32, gk32, gT32) = r[lbfe.FP64], r[lbfe.FP32]
    assert abs(L32 / L - 1) < 1e-4 and abs(gk32 / gk - 1) < 1e-4 and abs(gT32 / gT - 1) < 1e-4
    assert np.abs(g32 - g).max() < 1e-4 * np.abs(g).max()


def test_adjoint_rejects_bad_rho0_and_pressure_tensor():
    gc, _, rho0, sf = _setup(12, 10, lbfe.IMPROVED, lbfe.BGK)
    bad = rho0.copy()
    bad[2, 3] = -1.0
    with pytest.raises(lbfe.LBError):
        lbfe.Lattice([gc], precision=lbfe.FP64).adjoint(0, bad, 5, 0)
    for scheme in (lbfe.STANDARD_PT, lbfe.IMPROVED_SMOOTH):
        other, _, _, _ = _setup(12, 10, scheme, lbfe.BGK)
        with pytest.raises(lbfe.LBError):
            lbfe.Lattice([other], precision=lbfe.FP64).adjoint(0, rho0, 5, 0)


def test_gpu_adjoint_matches_oracle_droplet_64():
    """A longer horizon on the droplet shape of the differentiation workload
    (64^2, radius 16, 200 steps, u window of 20, checkpoints every 20) against
    the oracle's reverse sweep."""
    gc, oc, _, _ = _setup(64, 64, lbfe.IMPROVED, lbfe.BGK)
    e = thermo.vdw_paper()
    _, rg, rl = thermo.maxwell_reduced(e, 0.8)
    rho0 = inputs.droplet(64, 64, 16.0, rl, rg)
    sf = np.zeros((64, 64))
    sf[:8, :8] = sf[:8, -8:] = sf[-8:, :8] = sf[-8:, -8:] = 1e-2 / 256
    lat = lbfe.Lattice([gc], precision=lbfe.FP64)
    L, g, gk, gT = lat.adjoint(0, rho0, 200, 180, sf, 20)
    Lo, go, gko, gTo = O.adjoint(oc, rho0, 200, 180, sf)
    assert abs(L / Lo - 1) < 1e-9
    assert abs(gk / gko - 1) < 1e-8 and abs(gT / gTo - 1) < 1e-8
    np.testing.assert_allclose(g, go, rtol=0, atol=1e-8 * np.abs(go).max())
