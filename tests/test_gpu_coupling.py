"""Coupling methods 1 and 2 of section 3.5.2 (explicit A1, A2 and total
absorption; Planck absorption at T_- or T_+) on the CUDA path (general stage
kernel) against the FP64 oracle: a flat box with a moving fluid (boosted
interaction), a static box, and the Kerr torus; FP64 at 1e-11 per intensity
and on u_g, FP32 storage at 1e-4 (floor 1e-3).  The oracle's two methods are
pinned to the paper's printed equations in test_oracle_coupling.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle
import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import workloads as W
from helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def flat_case(moving, index):
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + index))
    nx = (10, 6, 4)
    nc = int(np.prod(nx))
    cfg = W.base_config(4, nx, (0, 0, 0), tuple(1.0 / n for n in nx), (("periodic", "periodic"),) * 3)
    rho = np.exp(rng.normal(0.0, 0.5, nc))
    T = rng.uniform(0.5, 2.0, nc)
    ucon = W.static_ucon(nc)
    if moving:
        v = rng.uniform(-0.2, 0.2, (nc, 3))
        g = 1.0 / np.sqrt(1.0 - (v * v).sum(1))
        ucon = np.concatenate([g[:, None], g[:, None] * v], axis=1)
    f = dict(rho=rho, ug=rho * T / (W.GAMMA - 1.0), ucon=ucon, kappa=np.full(nc, 0.3), alpha_s=np.full(nc, 0.4),
             eta=np.ones(nc), I=W.planck(rng.uniform(0.5, 2.0, nc))[:, None] * (1.0 + 0.1 * rng.uniform(-1, 1, (nc, 162))))
    return cfg, f


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("case", ["static", "moving", "kerr"])
def test_coupling_method_parity(method, case):
    if case == "kerr":
        cfg, f = W.kerr(nr=24, nth=16, nph=1, n_geo=4, index=90 + method)
    else:
        cfg, f = flat_case(case == "moving", 92 + method)
    cfg = dict(cfg, coupling=method)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 3)
    assert ref["fails"] == 0
    out = run_gpu(cfg, f, dt, 3, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    o32 = run_gpu(cfg, f, dt, 3, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4


def test_reverse_mode_refuses_methods_1_and_2():
    cfg, f = flat_case(False, 95)
    st = rt.RadiationStep(rt.Grid(4), dict(cfg, coupling=1), precision="fp64")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    st.set_fluid(T(f["rho"]), T(f["ug"]), T(f["ucon"]), T(f["kappa"]), T(f["alpha_s"]), T(f["eta"]))
    st.set_intensity(T(f["I"]))
    with pytest.raises(rt.RTError) as e:
        st.step_record(1e-3, 1)
    assert e.value.status == 1
