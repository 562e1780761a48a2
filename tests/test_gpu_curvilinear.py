"""Rotating tetrads in flat space on the CUDA path (general stage kernel
with geometry tables): snake coordinates (App. A.1, section 4.6) and
Cartesian coordinates with the cylindrical tetrad (section 4.5), against the
FP64 oracle (<= 1e-11 per intensity, floor 1e-6) and against the
straight-line pins of test_oracle_curvilinear.py.  FP32 storage: the packet
is a sharp peak in direction space, where the minimum-angle plane choice of
section 3.4 flips between near-tied planes under FP32 rounding (see the
kerr2d workload test); where it flips, the edge value moves by the
difference between two planes' reconstructions, a few per cent of the
peak.  Which planes flip depends on the FP32 rounding order: with the
general kernel's explicit multiply-adds the cylinder measures 2.9e-2 and
the snake 8.4e-3 (with the compiler's contraction, 8.4e-3 and below 1e-4).
Bar: 5e-2 per intensity (floor 1e-3), and the same straight-line bar as
FP64, which the flips do not move."""
import pytest

torch = pytest.importorskip("torch")
import curvilinear_cases as CC
import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import workloads as W
from helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


@pytest.mark.parametrize("fn,cells", [(CC.snake, 3.0), (CC.cylinder, 2.5)])
def test_rotating_tetrad_packet(fn, cells):
    cfg, f, dt, n, cerr = fn()
    ref = run_oracle(cfg, f, dt, n)
    out = run_gpu(cfg, f, dt, n, "fp64")
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert cerr(out["I"]) < cells * cfg["dx"][0]
    o32 = run_gpu(cfg, f, dt, n, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 5e-2
    assert cerr(o32["I"]) < cells * cfg["dx"][0]


def test_cylindrical_tetrad_refuses_the_axis():
    cfg = W.base_config(2, (8, 8, 1), (-1.0, -1.0, 0.0), (0.25, 0.25, 0.1),
                        (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                        coords="cart_cyl_tetrad")
    with pytest.raises(rt.RTError) as e:
        rt.RadiationStep(rt.Grid(2), cfg, precision="fp64")
    assert e.value.status == 1
