"""Row plans of the row-varying operator, checked on the host (no GPU).

wdb_vtheta_plan_check builds the per-output-row tap plan of Theta_K or Theta_K^T from the
oracle's kept taps (oracle.varying, Sec. 3.4 + 3.7) and runs one application with the kernel's
own index arithmetic and bounds checks; the result must equal the oracle's CSR product. The
cases cover every tap form (input finer, same level, coarser with phases), several levels,
rectangular images, and every output row without taps.
"""
import numpy as np
import pytest

from oracle import varying as V
from paper_1512_08401_gb300 import synthetic as S


@pytest.fixture(scope="module")
def wdb():
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


CASES = [((32, 32), "db4", 2, None), ((32, 32), "db2", 3, 8), ((32, 64), "db2", 3, 12), ((64, 32), "sym4", 2, 30),
         ((64, 64), "db1", 4, 30)]


@pytest.mark.parametrize("shape,wavelet,J,kn", CASES)
def test_plan_emulation_equals_oracle_products(wdb, shape, wavelet, J, kn):
    R, C = shape
    ps = S.varying_gaussian(R, 0.8, 2.5, 7)
    K = 10**12 if kn is None else kn * R * C
    th = V.build_varying_theta(ps, R, C, wavelet, J, K)
    t = th.taps
    x = np.random.default_rng(7).standard_normal(R * C)
    for tr, M in ((False, th.mat), (True, th.matT)):
        y = wdb.vtheta_plan_check(R, C, wavelet, J, t.a, t.py, t.b, t.qy, t.ox, t.v, x, transpose=tr)
        assert np.abs(y - M @ x).max() <= 1e-12 * max(1.0, np.abs(M @ x).max())


def test_plan_check_rejects_bad_taps(wdb):
    R = C = 32
    with pytest.raises(wdb.WdbError) as e:
        wdb.vtheta_plan_check(R, C, "db2", 2, [0], [0], [1], [0], [99], [1.0], np.zeros(R * C))
    assert e.value.status == 1
    with pytest.raises(wdb.WdbError) as e:
        wdb.vtheta_plan_check(R, C, "db2", 2, [0], [0], [77], [0], [0], [1.0], np.zeros(R * C))
    assert e.value.status == 1
    with pytest.raises(wdb.WdbError) as e:
        wdb.vtheta_plan_check(64, 4096, "db2", 2, [], [], [], [], [], [], np.zeros(64 * 4096))
    assert e.value.status == 7
