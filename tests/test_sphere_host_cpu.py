"""The library's host code for the G-sphere and the default FFT box, on the CPU (no context, no
device): bit-exact against the oracle's brute-force enumeration, and the exact counts of the
stored values.  The same code runs inside kss_setup, whose device-side maps the GPU tests check
against the oracle as well."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def _triclinic():
    lat = np.array([[7.1, 0.0, 0.0], [1.3, 6.4, 0.0], [-0.9, 0.7, 8.2]])
    return lat, 4.5, [(0.25, -0.25, 0.25), (0.1, 0.37, -0.41)]


def test_exact_counts(lib):
    c1, c2 = W.config1(), W.config2()
    assert K.kss_sphere_host(c1.lattice, c1.ecut, (0, 0, 0)).shape == (1503, 3)
    for k in c2.kpts:
        assert K.kss_sphere_host(c2.lattice, c2.ecut, k).shape == (34181, 3)


def test_bit_exact_against_oracle(lib):
    cases = [(W.config1().lattice, W.config1().ecut, (0.0, 0.0, 0.0))]
    c2 = W.config2()
    cases += [(c2.lattice, c2.ecut, k) for k in c2.kpts[:2]]
    lat, ec, ks = _triclinic()
    cases += [(lat, ec, k) for k in ks]
    for s in W.config4()[::6]:
        cases += [(s.lattice, s.ecut, k) for k in s.kpts[:2]]
    for lat, ec, k in cases:
        got = K.kss_sphere_host(lat, ec, k)
        ref = O.enumerate_sphere(np.asarray(lat, np.float64), ec, np.asarray(k, np.float64))
        assert np.array_equal(got.astype(np.int64), np.asarray(ref, np.int64)), (ec, k)


def test_default_box_matches_oracle(lib):
    systems = W.config4()[::4]
    for s in systems:
        assert s.fft_box is None
        assert K.kss_default_box(s.lattice, s.ecut, s.kpts) == O.system_box(s)
    lat, ec, ks = _triclinic()
    spheres = [O.enumerate_sphere(lat, ec, np.asarray(k, np.float64)) for k in ks]
    assert K.kss_default_box(lat, ec, ks) == O.default_box(spheres)
    c2 = W.config2()  # its literal box is 96^3; the default rule gives 4 * 20 + 1 = 81 = 3^4
    assert K.kss_default_box(c2.lattice, c2.ecut, c2.kpts) == (81, 81, 81)


def test_rejections(lib):
    lat = np.ascontiguousarray(np.eye(3).reshape(9) * 6.0)
    k = np.zeros(3)
    n = ctypes.c_int()
    L = lib
    assert L.kss_sphere_host(lat.ctypes.data, 0.0, k.ctypes.data, 0, ctypes.byref(n), None) == K.KSS_EINVAL
    assert L.kss_sphere_host(lat.ctypes.data, 2.0, k.ctypes.data, 0, None, None) == K.KSS_EINVAL
    bad = lat.copy()
    bad[4] = np.nan
    assert L.kss_sphere_host(bad.ctypes.data, 2.0, k.ctypes.data, 0, ctypes.byref(n), None) == K.KSS_EINVAL
    sing = lat.copy()
    sing[6:9] = sing[3:6]
    assert L.kss_sphere_host(sing.ctypes.data, 2.0, k.ctypes.data, 0, ctypes.byref(n), None) == K.KSS_EINVAL
    assert L.kss_sphere_host(lat.ctypes.data, 2.0, k.ctypes.data, 0, ctypes.byref(n), None) == K.KSS_OK
    assert n.value > 1
    small = np.zeros((n.value - 1, 3), np.int32)
    assert L.kss_sphere_host(lat.ctypes.data, 2.0, k.ctypes.data, n.value - 1, ctypes.byref(n),
                             small.ctypes.data) == K.KSS_EINVAL
    box = np.zeros(3, np.int32)
    assert L.kss_default_box(lat.ctypes.data, 2.0, 0, k.ctypes.data, box.ctypes.data) == K.KSS_EINVAL
    kn = np.array([np.nan, 0.0, 0.0])
    assert L.kss_default_box(lat.ctypes.data, 2.0, 1, kn.ctypes.data, box.ctypes.data) == K.KSS_EINVAL
