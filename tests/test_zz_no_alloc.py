"""rt_cfl_dt_noalloc (an interface with no counterpart in the paper) against
rt_cfl_dt through the C ABI: same bound on two calls in a row, for flat and
Kerr-Schild geometry, and the size limit of its static scratch array.

This file is collected last on purpose: the entry point must give the same
result in a fresh process and after every other test has used the device.
"""
import pytest

from helpers import rel_err

pytestmark = pytest.mark.gpu

# FP64 parity tolerance of the step tests; the bound is computed in FP64 on
# both sides
TOL = 1e-11


def _ctx(cfg, n_geo):
    import paper_2508_15532_b300 as rt
    return rt.RadiationStep(rt.Grid(n_geo), cfg, precision="fp32")


@pytest.mark.parametrize("kind", ["flat", "kerr2d", "kerr3d_pole"])
def test_noalloc_cfl_matches_allocating_entry_point(kind):
    from paper_2508_15532_b300 import workloads as W
    if kind == "flat":
        cfg, _ = W.flat3d(N=16, n_geo=4, index=301, with_intensity=False)
        ng = 4
    elif kind == "kerr2d":
        cfg, _ = W.kerr(nr=96, nth=64, nph=1, n_geo=4, index=302)
        ng = 4
    else:
        cfg, _ = W.kerr(nr=64, nth=48, nph=8, n_geo=2, index=303)
        ng = 2
    st = _ctx(cfg, ng)
    for cfl in (0.4, 0.25):                # two calls in a row share the scratch
        ref = st.cfl_dt(cfl)
        got = st.cfl_dt_noalloc(cfl)
        assert ref > 0.0
        assert rel_err([got], [ref])[0] <= TOL, (kind, cfl, got, ref)


def test_noalloc_cfl_rejects_sizes_beyond_its_scratch():
    import paper_2508_15532_b300 as rt
    from paper_2508_15532_b300 import workloads as W
    # 512 x 256 points x 162 directions = 21,233,664 > 16,777,216 items
    cfg, _ = W.kerr(nr=512, nth=256, nph=1, n_geo=4, index=304)
    st = _ctx(cfg, 4)
    with pytest.raises(rt.RTError, match="static scratch limit"):
        st.cfl_dt_noalloc(0.4)
    assert st.cfl_dt(0.4) > 0.0            # the allocating entry point still serves it
