"""Host-side helpers of bench.py on CPU: the droplet-shape diagnostics of the
sliding-walls workload and the core-list parser of the host binding."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _ellipse(nx, ny, cx, cy, a, b, rho_l=6.0, rho_g=1.0):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx = (x - cx + nx / 2) % nx - nx / 2
    inside = (dx / a) ** 2 + ((y - cy) / b) ** 2 < 1.0
    return np.where(inside, rho_l, rho_g)


def test_droplet_shape_of_a_circle_and_an_ellipse():
    cx, cy, ar = bench._droplet_shape(_ellipse(120, 120, 40.0, 60.0, 20.0, 20.0), 1.0)
    assert abs(cx - 40.0) < 0.05 and abs(cy - 60.0) < 0.05 and abs(ar - 1.0) < 0.01
    # an ellipse of axes 24 x 16: the inertia-tensor aspect ratio is a / b
    _, _, ar = bench._droplet_shape(_ellipse(120, 120, 60.0, 60.0, 24.0, 16.0), 1.0)
    assert abs(ar - 1.5) < 0.02


def test_droplet_shape_across_the_periodic_edge():
    """A droplet centred on x = 2 straddles the periodic edge in x: the
    circular mean keeps its centroid and its shape."""
    cx, cy, ar = bench._droplet_shape(_ellipse(120, 120, 2.0, 50.0, 15.0, 15.0), 1.0)
    assert min(abs(cx - 2.0), abs(cx - 122.0)) < 0.05 and abs(cy - 50.0) < 0.05 and abs(ar - 1.0) < 0.01


def test_cpulist_parser():
    assert bench._parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._parse_cpulist("5") == {5}
    assert bench._parse_cpulist("") == set()


def test_cpulist_format_round_trip():
    assert bench._format_cpulist({0, 1, 2, 3, 64, 65, 66, 67, 9}) == "0-3,9,64-67"
    assert bench._parse_cpulist(bench._format_cpulist({5, 7, 8, 9})) == {5, 7, 8, 9}


def test_gpu_ids_follow_the_pci_location_not_the_cuda_ordinal():
    """Under CUDA_VISIBLE_DEVICES=3, cuda:0 is the fourth GPU of the node:
    the ids used for nvidia-smi and the sysfs topology come from the
    device's PCI location, whatever its CUDA ordinal."""
    class Props:  # what torch reports for cuda:0 when it is the GPU at 0000:1B:00.0
        pci_domain_id, pci_bus_id, pci_device_id = 0, 0x1B, 0

    smi, sysfs = bench._pci_ids(Props())
    assert smi == "00000000:1B:00.0"
    assert sysfs == "0000:1b:00.0"


def test_scheme_option_names_library_schemes():
    """Every --scheme choice names a scheme code of the binding, and the
    workload text that the line reports names it."""
    from paper_2008_01473_gb300 import lbfe

    codes = {getattr(lbfe, attr) for attr, _ in bench.SCHEMES.values()}
    assert codes == {lbfe.STANDARD, lbfe.IMPROVED, lbfe.STANDARD_PT, lbfe.IMPROVED_SMOOTH}
    assert "improved scheme" in bench.WORKLOAD  # the text the option replaces
