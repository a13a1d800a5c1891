"""Host logic of the tile planner (no GPU): plans of Theta_K and Theta_K^T built by libwdb for
operators from the oracle, checked by wdb_tile_plan_check -- every output produced exactly
once, staged regions and tap areas inside the staging buffer, every staged read inside its
pair's region, and the conditions of split tiles, super tiles, grouped items and 16-byte
staging -- over the planner's parameter space."""
import numpy as np
import pytest

from paper_1512_08401_gb300 import synthetic

from oracle_cases import build_case, taps_arrays

CASES = {
    "gauss64_J3": (synthetic.gaussian_psf(1.5, 9), 64, 64, 3),
    "motion64_J3": (synthetic.motion_line_psf(7, 0.9), 64, 64, 3),
    "ragged48x80_J3": (synthetic.gaussian_psf(1.2, 7), 48, 80, 3),
    "gauss128_J4": (synthetic.gaussian_psf(2.0, 15), 128, 128, 4),
    "tiny16_J4": (synthetic.gaussian_psf(1.0, 5), 16, 16, 4),
}

CONFIGS = [
    dict(),
    dict(smem_budget=8192, cap_share=1.0, split_share=0.05),
    dict(smem_budget=24576, cap_share=4.0, split_share=1.0),
    dict(super_tiles=True),
    dict(smem_budget=49152, cap_share=4.0, super_tiles=True),
    dict(smem_budget=98304, cap_share=4.0),
    dict(esize=8),
    dict(esize=8, smem_budget=8192),
    dict(ctas=8, cap_share=1.0),
    dict(grouped=True),
    dict(grouped=True, smem_budget=49152, cap_share=4.0),
    dict(grouped=True, smem_budget=8192, cap_share=1.0),
    dict(grouped=True, esize=8),
]


@pytest.fixture(scope="module")
def wdb():
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    psf, nr, nc, J = CASES[request.param]
    c = build_case(psf, nr, nc, J, 30 * nr * nc, np.zeros((nr, nc)))
    return request.param, nr, nc, J, c, taps_arrays(c.th)


@pytest.mark.parametrize("transpose", [False, True])
def test_plans_keep_their_invariants(wdb, case, transpose):
    name, nr, nc, J, c, taps = case
    macs = set()
    for cfg in CONFIGS:
        s = wdb.tile_plan_check(nr, nc, J, *taps, transpose=transpose, **cfg)   # raises on a broken invariant
        assert s["items"] > 0 and s["pairs"] > 0 and s["batches"] >= 1
        macs.add(s["macs"])
        if not cfg.get("super_tiles"):
            assert s["super_subbands"] == 0
        if not cfg.get("split_share"):
            assert s["split_tiles"] == 0
        if cfg.get("grouped"):
            assert s["groups"] == J and s["super_subbands"] == 0   # A_J with level J, then J - 1 levels
        else:
            assert s["groups"] == 0
    # the multiply-adds per application depend on the operator, not on the plan; they count
    # every kept entry once (up pairs are padded to their fullest phase)
    assert len(macs) == 1
    assert c.th.K_eff <= macs.pop() <= 2 * c.th.K_eff


def test_split_and_super_tiles_are_used(wdb, case):
    name, nr, nc, J, c, taps = case
    if name != "gauss128_J4":
        pytest.skip("covered on the 128^2 operator")
    for tr in (False, True):
        assert wdb.tile_plan_check(nr, nc, J, *taps, transpose=tr, smem_budget=8192, cap_share=1.0,
                                   split_share=0.05)["split_tiles"] > 0
        assert wdb.tile_plan_check(nr, nc, J, *taps, transpose=tr, super_tiles=True)["super_subbands"] > 0


def test_bad_arguments(wdb, case):
    name, nr, nc, J, c, taps = case
    if name != "gauss64_J3":
        pytest.skip("once")
    a, b, oy, ox, v = taps
    with pytest.raises(wdb.WdbError):
        wdb.tile_plan_check(nr, nc, J, a, b, oy, ox, v, esize=2)
    with pytest.raises(wdb.WdbError):
        wdb.tile_plan_check(nr, nc, J, a, b, oy, ox, v, smem_budget=98305)
    bad = a.copy()
    bad[0] = 3 * J + 1   # one past the last subband
    with pytest.raises(wdb.WdbError):
        wdb.tile_plan_check(nr, nc, J, bad, b, oy, ox, v)
    with pytest.raises(wdb.WdbError):
        wdb.tile_plan_check(nr + 1, nc, J, a, b, oy, ox, v)   # not divisible by 2^J


@pytest.mark.parametrize("blur", ["gaussian", "motion"])
@pytest.mark.parametrize("transpose", [False, True])
def test_headline_operator_plans_keep_their_invariants(wdb, blur, transpose):
    """The two 1024^2 operators the headline bench runs (J = 5, K = 30N; taps from the oracle's
    records) under every planner configuration: the same invariants, and the same
    multiply-adds per application whatever the plan."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    d = np.load(os.path.join(root, "oracle", "data", f"theta_1024_{blur}_k30.npz"))
    n, J = int(d["n"]), int(d["levels"])
    taps = (d["a"].astype(np.int32), d["b"].astype(np.int32), d["oy"].astype(np.int32), d["ox"].astype(np.int32),
            d["v"].astype(np.float64))
    macs = set()
    for cfg in CONFIGS:
        s = wdb.tile_plan_check(n, n, J, *taps, transpose=transpose, **cfg)
        assert s["items"] > 0 and s["batches"] >= 1
        if cfg.get("grouped"):
            assert s["groups"] == J
        macs.add(s["macs"])
    assert len(macs) == 1
    assert int(d["K_eff"]) <= macs.pop() <= 2 * int(d["K_eff"])
