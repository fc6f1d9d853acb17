"""The row kernel for short periodic lattices (ny <= 16; the standard
scheme with either force form, the improved scheme, and the improved scheme
with the averaged correction): one thread per node of a whole-height strip,
the stages separated by block
barriers. FP64 against the oracle (1e-11), FP32 against the sliding-window
kernels that run the same lattices with the row kernel off (LBFE_ROWS=0) to
FP32 rounding, its work-list (one item per strip of at most 56, 58 or 60
columns), lattices of one and two rows per thread in one
launch, a batch that mixes it with the other kernels, the variable
viscosity, and the instability flag."""
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


def _case(nx, ny, scheme, collision, eos="vdw", nu=0.0, t=0.85):
    e = thermo.vdw_paper() if eos == "vdw" else thermo.EOS(thermo.CS, 9 / 392, 9 / 98)
    T, rg, rl = thermo.maxwell_reduced(e, t)
    kw = dict(nx=nx, ny=ny, scheme=scheme, collision=collision, eos=e.kind, a=e.a, b=e.b, R=1.0, T=T,
              kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1, nu=nu)
    return kw, rg, rl


def _rho0(nx, ny, rl, rg, seed):
    """A tilted liquid slab with noise and wide interfaces (the standard
    scheme blows up within 25 steps from sharper ones): gradients in x and
    y at every row."""
    y, x = np.mgrid[0:ny, 0:nx]
    d = np.cos(2 * np.pi * (x / nx + y / ny))
    rho = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh(1.5 * d)
    return rho + 1e-3 * (2 * inputs.splitmix_uniform(seed, 0, nx, ny) - 1)


def _flow(nx, ny):
    return (0.01 * (2 * inputs.splitmix_uniform(2, 0, nx, ny) - 1),
            0.01 * (2 * inputs.splitmix_uniform(3, 0, nx, ny) - 1))


def _maxerr(m, ref):
    return max(np.abs(m["rho"] - ref.rho).max(), np.abs(m["ux"] - ref.ux).max(), np.abs(m["uy"] - ref.uy).max())


def _strips(nx, scheme):
    w = {lbfe.IMPROVED: 58, lbfe.IMPROVED_SMOOTH: 56}.get(scheme, 60)
    return (nx + w - 1) // w


@pytest.mark.parametrize("scheme", [lbfe.STANDARD, lbfe.IMPROVED, lbfe.STANDARD_PT, lbfe.IMPROVED_SMOOTH])
@pytest.mark.parametrize("collision", [lbfe.BGK, lbfe.MRT])
@pytest.mark.parametrize("shape", [(64, 8), (130, 13), (37, 3), (203, 16), (11, 5)])
def test_fp64_rows_kernel_matches_oracle(scheme, collision, shape):
    """25 FP64 steps from a tilted slab with noise and an initial flow: rho,
    u and mu_c equal the oracle's to 1e-11; the work-list holds one item per
    strip (the row kernel's), several strips on the wider lattices, one
    strip wider than the lattice on the narrow ones. With the averaged
    correction the 5 x 5 stencil's rows wrap within heights of 3 and 5."""
    nx, ny = shape
    kw, rg, rl = _case(nx, ny, scheme, collision)
    rho0 = _rho0(nx, ny, rl, rg, 7)
    ux0, uy0 = _flow(nx, ny)
    lat = lbfe.Lattice([lbfe.Case(**kw)], precision=lbfe.FP64)
    lat.init_fields(0, rho0, ux0, uy0)
    lat.step(25)
    assert lat.worklist()[1] == _strips(nx, scheme)
    m = lat.moments(0)
    _, st = lat.reductions()
    lat.close()
    assert st[0] == 0
    oc = O.Case(**kw)
    f = O.init(oc, rho0, ux0, uy0)
    assert O.step(oc, f, 25) == 25
    ref = O.fields(oc, f)
    assert _maxerr(m, ref) < 1e-11
    assert np.abs(m["mu"] - ref.mu).max() < 1e-11


@pytest.mark.parametrize("eos,nu", [("cs", 0.0), ("vdw", 0.05)])
def test_fp64_rows_kernel_eos_and_variable_viscosity(eos, nu):
    """The Carnahan-Starling equation of state and the density-dependent
    viscosity (nu > 0) on the row kernel, against the oracle."""
    nx, ny = 96, 12
    for scheme in (lbfe.STANDARD, lbfe.IMPROVED, lbfe.STANDARD_PT, lbfe.IMPROVED_SMOOTH):
        kw, rg, rl = _case(nx, ny, scheme, lbfe.MRT, eos=eos, nu=nu)
        rho0 = _rho0(nx, ny, rl, rg, 11)
        lat = lbfe.Lattice([lbfe.Case(**kw)], precision=lbfe.FP64)
        lat.init_fields(0, rho0)
        lat.step(20)
        m = lat.moments(0)
        lat.close()
        oc = O.Case(**kw)
        f = O.init(oc, rho0)
        assert O.step(oc, f, 20) == 20
        assert _maxerr(m, O.fields(oc, f)) < 1e-11


def _run(cases, rhos, steps, precision, rows, monkeypatch):
    monkeypatch.setenv("LBFE_ROWS", "1" if rows else "0")
    lat = lbfe.Lattice(cases, precision=precision)
    for i, r in enumerate(rhos):
        lat.init_fields(i, r)
    lat.step(steps)
    out = [lat.moments(i) for i in range(len(cases))]
    items = lat.worklist()[1]
    _, st = lat.reductions()
    lat.close()
    assert (st == 0).all()
    return out, items


@pytest.mark.parametrize("scheme", [lbfe.STANDARD, lbfe.IMPROVED, lbfe.STANDARD_PT, lbfe.IMPROVED_SMOOTH])
def test_fp32_rows_kernel_matches_sliding_window(scheme, monkeypatch):
    """FP32: one launch over lattices of one row per thread (ny <= 8) and
    two (ny 9 ... 16) of uneven widths; after 40 steps rho (about 0.8 to 6.8)
    and u agree with the sliding-window kernels to the FP32 rounding that 40
    steps accumulate (1e-4 and 1e-5 absolute), and rho with the FP64 oracle
    to the same bound."""
    shapes = [(1024, 8), (200, 16), (61, 9), (64, 4)]
    cases, rhos, kws = [], [], []
    for k, (nx, ny) in enumerate(shapes):
        kw, rg, rl = _case(nx, ny, scheme, lbfe.BGK, t=0.85)
        kws.append(kw)
        cases.append(lbfe.Case(**kw))
        rhos.append(_rho0(nx, ny, rl, rg, 30 + k))
    rows, n_rows = _run(cases, rhos, 40, lbfe.FP32, True, monkeypatch)
    window, _ = _run(cases, rhos, 40, lbfe.FP32, False, monkeypatch)
    assert n_rows == sum(_strips(nx, scheme) for nx, _ in shapes)
    for k, (a, b) in enumerate(zip(rows, window)):
        for key in ("rho", "ux", "uy"):
            assert np.abs(a[key] - b[key]).max() < (1e-4 if key == "rho" else 1e-5), (k, key)
    oc = O.Case(**kws[2])
    f = O.init(oc, rhos[2])
    assert O.step(oc, f, 40) == 40
    assert np.abs(rows[2]["rho"] - O.fields(oc, f).rho).max() < 1e-4


@pytest.mark.parametrize("precision", [lbfe.FP64, lbfe.FP32])
def test_rows_kernel_in_a_batch(precision, monkeypatch):
    """A handle whose short periodic lattices run on the row kernel next to
    a taller lattice and a walled one on the other kernels: every case gives
    the bits it gives alone."""
    kw1, rg, rl = _case(120, 8, lbfe.IMPROVED, lbfe.MRT)
    kw2, _, _ = _case(48, 40, lbfe.IMPROVED, lbfe.MRT)
    kw3, _, _ = _case(64, 12, lbfe.STANDARD, lbfe.BGK)
    kw4 = dict(kw2, walls=1, wall_u=0.02, rho_wall=rg)
    kws = [kw1, kw2, kw3, kw4]
    rhos = [_rho0(k["nx"], k["ny"], rl, rg, 50 + i) for i, k in enumerate(kws)]
    batch, _ = _run([lbfe.Case(**k) for k in kws], rhos, 30, precision, True, monkeypatch)
    for i, k in enumerate(kws):
        (alone,), _ = _run([lbfe.Case(**k)], [rhos[i]], 30, precision, True, monkeypatch)
        for key in ("rho", "ux", "uy", "mu"):
            assert np.array_equal(batch[i][key], alone[key]), (i, key)


def test_rows_kernel_flags_and_freezes_an_unstable_case():
    """Carnahan-Starling a=1, b=4 at 0.5 T_c on a 64 x 8 strip blows up
    within a few steps: the row kernel flags it and returns at once for it
    from then on (its populations stay as they are)."""
    e = thermo.cs_unit()
    T, rg, rl = thermo.maxwell_reduced(e, 0.5)
    bad = lbfe.Case(nx=64, ny=8, scheme=lbfe.IMPROVED, collision=lbfe.BGK, eos=lbfe.CS, a=1.0, b=4.0, T=T,
                    kappa=0.02, tau_v=1.0)
    lat = lbfe.Lattice([bad], precision=lbfe.FP64)
    lat.init_fields(0, inputs.slab(64, 8, rl, rg))
    lat.step(50)
    _, st = lat.reductions()
    assert st[0] == 3
    frozen = lat.save(0)[16:]
    lat.step(16)  # even: the buffers swap every step and keep its last two states
    assert lat.save(0)[16:] == frozen
    lat.close()


def test_persistent_mode_takes_the_lattices_off_the_row_kernel():
    """lb_launch_mode(1) moves the short lattices to the persistent kernel's
    work-list (a single group) and mode 0 back to the row kernel; the state
    carries over and each mode's steps match the oracle."""
    kw, rg, rl = _case(150, 8, lbfe.IMPROVED, lbfe.BGK)
    rho0 = _rho0(150, 8, rl, rg, 3)
    lat = lbfe.Lattice([lbfe.Case(**kw)], precision=lbfe.FP64)
    lat.init_fields(0, rho0)
    lat.step(10)
    assert lat.worklist()[1] == _strips(150, lbfe.IMPROVED)
    assert lat.launch_mode(1)
    lat.step(40)
    n_persist = lat.worklist()[1]
    assert not lat.launch_mode(0)
    assert lat.worklist()[1] == _strips(150, lbfe.IMPROVED)
    lat.step(10)
    m = lat.moments(0)
    lat.close()
    assert n_persist >= 1
    oc = O.Case(**kw)
    f = O.init(oc, rho0)
    assert O.step(oc, f, 60) == 60
    assert _maxerr(m, O.fields(oc, f)) < 1e-11
