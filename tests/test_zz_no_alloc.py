"""lb_fields_static, the field-export and reduction pass that allocates
nothing, against the handle-based lb_moments / lb_reductions.

The static entry point serves callers that cannot give the library device
memory (plug-ins inside applications that own every allocation, code where
cudaMalloc would synchronise or is not allowed). Its scratch is a fixed array
inside the library shared by all calls on a device, so this test calls it
twice in a row, on two different cases, and checks each result against the
existing entry points. It runs alone or after the rest of the suite.
"""
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


def _reference_and_pops(case, rho0, steps, precision):
    """Existing path: lb_moments / lb_reductions of a handle; plus the state's
    stored populations uploaded to a device tensor in the snapshot layout."""
    import torch

    lat = lbfe.Lattice([case], precision=precision)
    lat.init_fields(0, rho0)
    lat.step(steps)
    ref = lat.moments(0)
    red, st = lat.reductions()
    snap = lat.save(0)
    rho_ref = float(np.frombuffer(snap[8:16], dtype=np.float64)[0])
    dt = np.float32 if precision == lbfe.FP32 else np.float64
    pops = torch.from_numpy(np.frombuffer(snap[16:], dtype=dt).copy()).cuda()
    lat.close()
    return ref, red[0], pops, rho_ref


def _static(case, precision, pops, rho_ref):
    import torch

    sh = (case.ny, case.nx)
    out = {k: torch.full(sh, np.nan, dtype=torch.float64, device="cuda") for k in ("rho", "ux", "uy", "mu")}
    red = torch.full((5,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cs = case.cstruct()
    rc = lbfe.lib().lb_fields_static(C.byref(cs), precision, C.c_void_p(pops.data_ptr()), rho_ref,
                                     *[C.c_void_p(out[k].data_ptr()) for k in ("rho", "ux", "uy", "mu")],
                                     C.c_void_p(red.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, red.cpu().numpy()


def _case(nx, ny, scheme, eos, t):
    e = thermo.vdw_paper() if eos == lbfe.VDW else thermo.EOS(thermo.CS, 9 / 392, 9 / 98)
    T, rg, rl = thermo.maxwell_reduced(e, t)
    c = lbfe.Case(nx=nx, ny=ny, scheme=scheme, collision=lbfe.MRT, eos=eos, a=e.a, b=e.b, T=T, kappa=0.02,
                  tau_v=0.8)
    return c, inputs.droplet(nx, ny, 0.3 * min(nx, ny), rl, rg, width=4.0, noise=1e-3, seed=4)


def test_static_matches_handle_path_two_calls():
    """Calls in a row (a larger FP32 improved case, a smaller FP64 standard
    one, then an FP64 case of the averaged-correction scheme) each equal
    lb_moments and lb_reductions within 1e-12."""
    runs = [(_case(300, 200, lbfe.IMPROVED, lbfe.VDW, 0.8), lbfe.FP32, 30),
            (_case(97, 61, lbfe.STANDARD, lbfe.CS, 0.9), lbfe.FP64, 25),
            (_case(64, 40, lbfe.IMPROVED_SMOOTH, lbfe.VDW, 0.7), lbfe.FP64, 20)]
    for (case, rho0), prec, steps in runs:
        ref, red_ref, pops, rho_ref = _reference_and_pops(case, rho0, steps, prec)
        got, red = _static(case, prec, pops, rho_ref)
        for k in ("rho", "ux", "uy", "mu"):
            np.testing.assert_allclose(got[k], ref[k], rtol=0, atol=1e-12)
        assert abs(red[0] / red_ref[0] - 1) < 1e-12
        assert abs(red[1] - red_ref[1]) <= 1e-12 * max(1.0, abs(red_ref[1]))
        assert abs(red[2] - red_ref[2]) < 1e-12
        assert red[3] == 0.0 and red[4] == 0.0


def test_static_allocates_nothing_and_reduces_without_field_outputs():
    """The contract itself: the device's free memory is the same before and
    after a call (the first call on the device may load the library's module,
    so the measured call is the second one), and a call with every field
    output NULL still writes the reductions, equal to lb_reductions."""
    import torch

    (case, rho0), prec, steps = _case(200, 150, lbfe.IMPROVED, lbfe.VDW, 0.8), lbfe.FP32, 20
    ref, red_ref, pops, rho_ref = _reference_and_pops(case, rho0, steps, prec)
    red = torch.full((5,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cs = case.cstruct()

    def call():
        rc = lbfe.lib().lb_fields_static(C.byref(cs), prec, C.c_void_p(pops.data_ptr()), rho_ref, None, None, None,
                                         None, C.c_void_p(red.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    r = red.cpu().numpy()
    assert abs(r[0] / red_ref[0] - 1) < 1e-12 and abs(r[2] - red_ref[2]) < 1e-12 and r[4] == 0.0


def test_static_rejects_oversized_case():
    import torch

    big = lbfe.Case(nx=1024, ny=512)  # 524288 nodes > LB_STATIC_MAX_NODES
    pops = torch.zeros(8, dtype=torch.float32, device="cuda")
    red = torch.zeros(5, dtype=torch.float64, device="cuda")
    cs = big.cstruct()
    rc = lbfe.lib().lb_fields_static(C.byref(cs), lbfe.FP32, C.c_void_p(pops.data_ptr()), 1.0, None, None, None,
                                     None, C.c_void_p(red.data_ptr()), None)
    assert rc == 1
    wide = lbfe.Case(nx=8192, ny=4)
    cs = wide.cstruct()
    rc = lbfe.lib().lb_fields_static(C.byref(cs), lbfe.FP32, C.c_void_p(pops.data_ptr()), 1.0, None, None, None,
                                     None, C.c_void_p(red.data_ptr()), None)
    assert rc == 1
