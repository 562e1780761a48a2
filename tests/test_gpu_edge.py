"""Edge and degenerate cases of the CUDA radiation step against the FP64
oracle: inactive axes (1D and 2D boxes, which select other brick shapes),
the coarsest geodesic grid (12 directions), cells below the interaction's
density floor (vacuum faces with tau = 0), and error reporting at the C ABI.

Bars as in the other parity tests: FP64 1e-11 per intensity, FP32 1e-4
(floor 1e-3 of the largest intensity)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle
import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import workloads as W
from helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def box(nx, n_geo=2, index=70, vacuum_frac=0.0):
    """flat3d-like fields on an arbitrary periodic box (axes of one cell are inactive)."""
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + index))
    nc = int(np.prod(nx))
    nd = 10 * n_geo * n_geo + 2
    cfg = W.base_config(n_geo, nx, (0, 0, 0), tuple(1.0 / max(n, 1) for n in nx), (("periodic", "periodic"),) * 3)
    rho = np.exp(rng.normal(0.0, 0.5, nc))
    if vacuum_frac > 0:
        rho[rng.random(nc) < vacuum_frac] = 1e-5          # below the 5e-4 floor: no interaction, tau = 0
    T = rng.uniform(0.5, 2.0, nc)
    f = dict(rho=rho, ug=rho * T / (W.GAMMA - 1.0), ucon=W.static_ucon(nc), kappa=np.full(nc, 1e-2),
             alpha_s=np.full(nc, 0.4), eta=np.ones(nc),
             I=W.planck(T)[:, None] * (1.0 + 0.1 * rng.uniform(-1, 1, (nc, nd))))
    return cfg, f


@pytest.mark.parametrize("nx", [(24, 1, 1), (12, 10, 1), (1, 12, 6), (9, 1, 7)])
def test_inactive_axes_fp64_and_fp32(nx):
    cfg, f = box(nx, index=71 + sum(nx))
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 4)
    out = run_gpu(cfg, f, dt, 4, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    o32 = run_gpu(cfg, f, dt, 4, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4


def test_twelve_directions():
    cfg, f = box((10, 8, 6), n_geo=1, index=80)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 3)
    assert rel_err(run_gpu(cfg, f, dt, 3, "fp64")["I"], ref["I"]).max() < 1e-11
    assert rel_err(run_gpu(cfg, f, dt, 3, "fp32")["I"], ref["I"], 1e-3).max() < 1e-4


def test_cells_below_density_floor():
    cfg, f = box((16, 8, 6), index=81, vacuum_frac=0.3)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 4)
    out = run_gpu(cfg, f, dt, 4, "fp64")
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    vac = f["rho"] < 5e-4
    assert np.array_equal(out["ug"][vac], f["ug"][vac])     # no exchange below the floor


def test_errors_at_the_boundary():
    g = rt.Grid(2)
    cfg, f = box((4, 4, 4), index=82)
    with pytest.raises(rt.RTError):
        rt.RadiationStep(g, dict(cfg, nx=(0, 4, 4)), precision="fp64")       # empty box
    st = rt.RadiationStep(g, cfg, precision="fp64")
    with pytest.raises(rt.RTError, match="RT_ESTATE"):
        st.step(1e-3, 1)                                                      # no fluid, no intensity
    with pytest.raises(rt.RTError):
        rt.Grid(3)                                                            # n must be a power of two
    g16 = rt.Grid(16)                                                         # 2562 directions
    cfg16, f16 = box((4, 4, 4), n_geo=16, index=83)
    st16 = rt.RadiationStep(g16, cfg16, precision="fp32")
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    st16.set_fluid(T(f16["rho"]), T(f16["ug"]), T(f16["ucon"]), T(f16["kappa"]), T(f16["alpha_s"]), T(f16["eta"]))
    st16.set_intensity(T(f16["I"]).float())
    with pytest.raises(rt.RTError, match="1024 directions"):
        st16.step(1e-3, 1)                                                    # beyond the stage kernel's limit
