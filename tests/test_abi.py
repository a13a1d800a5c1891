"""The C-ABI library builds, loads, exports every declared symbol and validates arguments
on the host (no GPU compute)."""
import ctypes as C

import numpy as np
import pytest

from oracle.wavelet import daubechies_lowpass, highpass_from_lowpass


@pytest.fixture(scope="module")
def wdb():
    from paper_1512_08401_gb300 import build, wdb as w
    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    w.lib()
    return w


def test_exports_every_header_symbol(wdb):
    names = wdb.header_functions()
    assert len(names) >= 20
    L = wdb.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_filters_derived_independently_match_oracle(wdb):
    for p in range(1, 11):
        h, g = wdb.wavelet_filters(f"db{p}")
        ref = daubechies_lowpass(p)
        assert np.abs(h - ref).max() < 1e-14
        assert np.abs(g - highpass_from_lowpass(ref)).max() < 1e-14


def test_symlets_derived_independently_match_oracle(wdb):
    from oracle.wavelet import symlet_lowpass
    for p in range(1, 11):
        h, g = wdb.wavelet_filters(f"sym{p}")
        ref = symlet_lowpass(p)
        assert np.abs(h - ref).max() < 1e-13, p
        assert np.abs(g - highpass_from_lowpass(ref)).max() < 1e-13, p


@pytest.mark.parametrize("kwargs,msg", [
    (dict(psf=np.ones((4, 5)) / 20), "odd"),
    (dict(psf=np.ones((65, 3)) / 195), "larger"),
    (dict(n=100), "divisible"),
    (dict(K=-1), "K"),
    (dict(wavelet="coif3"), "wavelet"),
    (dict(wavelet="sym11"), "sym"),
    (dict(wavelet="db11"), "db"),
    (dict(levels=0), "levels"),
])
def test_build_theta_rejects_bad_arguments(wdb, kwargs, msg):
    psf = kwargs.get("psf", np.ones((3, 3)) / 9)
    n = kwargs.get("n", 64)
    out = C.c_void_p()
    psf = np.ascontiguousarray(psf, dtype=np.float64)
    st = wdb.lib().wdb_build_theta(psf.ctypes.data_as(wdb.pd), psf.shape[0], psf.shape[1], n, n,
                                   kwargs.get("wavelet", "db4").encode(), kwargs.get("levels", 3),
                                   kwargs.get("K", 1000), 0, None, C.byref(out))
    assert st == 1, wdb.lib().wdb_last_error()
    assert msg.lower() in wdb.lib().wdb_last_error().decode().lower()
    assert out.value is None


def test_from_taps_rejects_bad_taps(wdb):
    out = C.c_void_p()
    a = np.array([0, 0], np.int32)
    b = np.array([0, 0], np.int32)
    oy = np.array([1, 1], np.int32)
    ox = np.array([2, 2], np.int32)
    v = np.array([1.0, 2.0])
    L = wdb.lib()
    st = L.wdb_theta_from_taps(32, 32, b"db4", 2, 2, a.ctypes.data_as(wdb.pi), b.ctypes.data_as(wdb.pi),
                               oy.ctypes.data_as(wdb.pi), ox.ctypes.data_as(wdb.pi), v.ctypes.data_as(wdb.pd),
                               None, C.byref(out))
    assert st == 1 and b"duplicate" in L.wdb_last_error()
    oy2 = np.array([1, 99], np.int32)
    st = L.wdb_theta_from_taps(32, 32, b"db4", 2, 2, a.ctypes.data_as(wdb.pi), b.ctypes.data_as(wdb.pi),
                               oy2.ctypes.data_as(wdb.pi), ox.ctypes.data_as(wdb.pi), v.ctypes.data_as(wdb.pd),
                               None, C.byref(out))
    assert st == 1 and b"range" in L.wdb_last_error()


def test_status_strings(wdb):
    L = wdb.lib()
    assert L.wdb_status_str(0) == b"ok"
    assert L.wdb_status_str(5) == b"timeout"
