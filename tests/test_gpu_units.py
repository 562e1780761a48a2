"""The section 3.5.1 unit scale through the CUDA path: the physical
equilibration of tests/test_units.py (gas at 4e7 K and radiation at 1e7 K in
1 g/cm^3, posed in code units by paper_2508_15532_b300/units.py) stepped by
the library in FP64 and FP32 storage reaches the cgs equilibrium temperature
(FP64 within 1e-9, FP32 within 1e-5) and matches the oracle run of the same
code-unit inputs at the FP64 bar."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from helpers import rel_err, run_gpu, run_oracle
import test_units as TU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_physical_equilibration_gpu():
    s, cfg, f, W_cgs = TU.physical_cell()
    T_eq = TU.equilibrium_K(W_cgs)
    ref = run_oracle(cfg, f, 2.0, 40)
    for prec, bar in (("fp64", 1e-9), ("fp32", 1e-5)):
        out = run_gpu(cfg, f, 2.0, 40, prec)
        assert out["fails"] == 0
        Tg = (cfg["gam"] - 1) * out["ug"][0] / f["rho"][0]
        assert abs(s.temperature_K(Tg) / T_eq - 1.0) < bar, prec
        if prec == "fp64":
            assert rel_err(out["I"], ref["I"]).max() < 1e-11
            assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
