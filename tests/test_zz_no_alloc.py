"""The allocation-free forward transform (wdb_dwt_noalloc) against wdb_dwt.

wdb_dwt_noalloc serves callers that cannot allocate device memory; its scratch lives in a
static device array shared by every call. Two calls in a row with different images must
each reproduce wdb_dwt (same kernels; the tolerance is the one the transform tests use),
so stale contents of the shared array cannot leak into a result. This file is collected
last on purpose: run alone in a fresh process, its first call also does the per-device
set-up.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wdb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


@pytest.mark.parametrize("n_rows,n_cols,J", [(1024, 1024, 5), (48, 80, 3)])
def test_noalloc_matches_dwt_twice(wdb, n_rows, n_cols, J):
    rng = np.random.default_rng(21)
    N = n_rows * n_cols
    for call in range(2):
        u = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
        ref = torch.zeros(N, device="cuda")
        got = torch.full((N,), float("nan"), device="cuda")
        wdb.dwt(u, ref, n_rows, n_cols, "db4", J)
        wdb.dwt_noalloc(u, got, n_rows, n_cols, "db4", J)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all(), f"call {call}"
        assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max(), f"call {call}"


def test_noalloc_second_call_leaves_device_memory_alone(wdb):
    """After the first call on this device (which may load the module holding the array),
    another call changes the device's free memory by nothing (cudaMemGetInfo), and its result
    agrees with the FP64 oracle's transform within the transform tests' tolerance."""
    from oracle import wavelet
    n_rows, n_cols, J = 256, 384, 4
    N = n_rows * n_cols
    rng = np.random.default_rng(22)
    img = rng.standard_normal((n_rows, n_cols))
    u = torch.from_numpy(img.astype(np.float32).ravel()).cuda()
    got = torch.zeros(N, device="cuda")
    wdb.dwt_noalloc(u, got, n_rows, n_cols, "db4", J)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    wdb.dwt_noalloc(u, got, n_rows, n_cols, "db4", J)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = wavelet.dwt2(img.astype(np.float32).astype(np.float64), "db4", J)
    a = got.cpu().numpy().astype(np.float64)
    assert np.abs(a - ref).max() <= 2e-6 * np.abs(ref).max()


def test_noalloc_rejects_oversize(wdb):
    u = torch.zeros(4, device="cuda")
    st = wdb.lib().wdb_dwt_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(u.data_ptr()), 4096, 4096, b"db4", 6, None)
    assert st == 1
    assert b"static array" in wdb.lib().wdb_last_error()
