"""Per-step statistics fused into the step kernels (lb_step_stats_*): the
mass, kinetic energy and max |u| recorded for every state a step starts from
agree with lb_reductions of the same state, for every step kernel (packed
FP32, one-column FP32 and FP64, the averaged correction, walls, the
Lax-Wendroff scheme, the row kernel of short periodic lattices), under graph replay and direct launches; the ring, the
restart at lb_init_fields and the persistent-launch exclusion behave as
include/lbfe.h states."""
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


def _cases():
    """Uneven lattices that take different kernels: packed (nx % 4 == 0),
    one-column (nx % 4 != 0), the averaged correction, walls, the
    Lax-Wendroff scheme and the row kernel (ny <= 16, two rows and one row
    per thread)."""
    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, 0.8)
    base = dict(eos=lbfe.VDW, a=e.a, b=e.b, R=1.0, T=T, kappa=0.02, tau_v=0.8)
    specs = [
        dict(nx=64, ny=48, scheme=lbfe.IMPROVED, collision=lbfe.MRT),
        dict(nx=41, ny=33, scheme=lbfe.STANDARD, collision=lbfe.BGK),
        dict(nx=96, ny=40, scheme=lbfe.IMPROVED_SMOOTH, collision=lbfe.MRT),
        dict(nx=48, ny=36, scheme=lbfe.IMPROVED, collision=lbfe.BGK, walls=1, wall_u=0.02, rho_wall=rg),
        dict(nx=40, ny=40, scheme=lbfe.LAX_WENDROFF, collision=lbfe.BGK, tau_v=1.0, lw_A=0.5, lw_B=-0.2),
        dict(nx=150, ny=12, scheme=lbfe.IMPROVED, collision=lbfe.MRT),
        dict(nx=72, ny=8, scheme=lbfe.STANDARD, collision=lbfe.BGK),
    ]
    cases, rho0s = [], []
    for k, kw in enumerate(specs):
        c = lbfe.Case(**{**base, **kw})
        cases.append(c)
        rho0s.append(inputs.droplet(c.nx, c.ny, 0.3 * min(c.nx, c.ny), rl, rg, width=3.0, noise=1e-3, seed=20 + k))
    return cases, rho0s


@pytest.mark.parametrize("precision", [lbfe.FP64, lbfe.FP32])
def test_step_stats_match_reductions(precision):
    cases, rho0s = _cases()
    n = 21  # two 8-step graphs and five direct launches
    lat = lbfe.Lattice(cases, precision=precision)
    ref = lbfe.Lattice(cases, precision=precision)
    for i, r in enumerate(rho0s):
        lat.init_fields(i, r)
        ref.init_fields(i, r)
    lat.attach_step_stats(64)
    lat.step(n)
    expect = []
    for _ in range(n):  # the same states, one step at a time (bit-identical whatever the work-list)
        out, st = ref.reductions()
        assert (st == 0).all()
        expect.append(out.copy())
        ref.step(1)
    expect = np.array(expect)  # [state, case, 5]
    tol = (1e-12, 1e-11, 1e-12) if precision == lbfe.FP64 else (2e-6, 1e-4, 1e-5)
    for i, c in enumerate(cases):
        first, rec = lat.step_stats(i)
        assert first == 0 and rec.shape == (n, 4), (i, first, rec.shape)
        assert (rec[:, 3] == c.nx * c.ny).all(), i
        for k in range(n):
            m, ke, um = expect[k, i, 0], expect[k, i, 1], expect[k, i, 2]
            assert abs(rec[k, 0] - m) <= tol[0] * m, (i, k, rec[k, 0], m)
            assert abs(rec[k, 1] - ke) <= tol[1] * ke + 1e-30, (i, k, rec[k, 1], ke)
            assert abs(rec[k, 2] - um) <= tol[2] * um + 1e-30, (i, k, rec[k, 2], um)
    # the states are the handle's own: the current state matches lb_reductions
    out, _ = lat.reductions()
    out_ref, _ = ref.reductions()
    assert np.array_equal(out[:, :3], out_ref[:, :3])
    lat.close()
    ref.close()


def test_step_stats_ring_restart_and_detach():
    cases, rho0s = _cases()
    cases, rho0s = cases[:2], rho0s[:2]
    lat = lbfe.Lattice(cases, precision=lbfe.FP32)
    for i, r in enumerate(rho0s):
        lat.init_fields(i, r)
    lat.step(3)  # the record starts at the state of the attach
    lat.attach_step_stats(8)
    lat.step(20)
    first, rec = lat.step_stats(0)
    assert first == 3 + 20 - 8 and rec.shape == (8, 4)
    with pytest.raises(lbfe.LBError):
        lat.step_stats(0, first - 1, 1)
    f1, row = lat.step_stats(1, first + 7, 1)
    assert f1 == first + 7 and np.array_equal(row[0], lat.step_stats(1)[1][7])
    # a new state restarts the case's record at state 0; the other case goes on
    lat.init_fields(0, rho0s[0])
    lat.step(2)
    assert lat.step_stats(0)[0] == 0 and lat.step_stats(0)[1].shape == (2, 4)
    assert lat.step_stats(1)[0] == 3 + 22 - 8
    lat.attach_step_stats(0)
    with pytest.raises(lbfe.LBError):
        lat.step_stats(0)
    lat.close()
    # persistent launch (a one-group handle): excluded while a buffer is attached
    solo = lbfe.Lattice(cases[:1], precision=lbfe.FP32)
    solo.init_fields(0, rho0s[0])
    solo.attach_step_stats(4)
    with pytest.raises(lbfe.LBError):
        solo.launch_mode(1)
    solo.attach_step_stats(0)
    assert solo.launch_mode(1)
    solo.close()


def test_step_stats_first_step_after_attach_records_from_the_tuner_state():
    """The autotuner's trial launches (first lb_step) record nothing: after
    lb_step(n) on a fresh handle exactly n states are recorded, and mass is
    conserved from one to the next to the FP32 partial-sum rounding."""
    cases, rho0s = _cases()
    lat = lbfe.Lattice(cases[:1], precision=lbfe.FP32)
    lat.init_fields(0, rho0s[0])
    lat.attach_step_stats(16)
    lat.step(10)
    first, rec = lat.step_stats(0)
    assert first == 0 and rec.shape == (10, 4)
    assert np.abs(rec[:, 0] / rec[0, 0] - 1).max() < 2e-6
    lat.close()
