"""The finer geodesic grid G3 of section 3.3 (n = 8: 642 directions, the grid
of the section 4.1 expansion test) on the CUDA path.  Beyond 256 directions
the general stage kernel runs one direction per thread in CTAs of up to 1024
threads with 1 x 1 bricks of 32, 16 or 8 cells (whatever shared memory
holds), so these cases cover that launch shape on every precision and
geometry: flat static and moving fluids, the Kerr-Schild torus (minimum-angle
reconstruction and angular fluxes over the finer rings) and the cylindrical
tetrad.  Bars as in the 162-direction parity tests: FP64 within 1e-11 of the
FP64 oracle per intensity (floor 1e-6 of the largest), FP32 storage within
1e-4 (floor 1e-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle
import closed_form_cases as CF
import curvilinear_cases as CC
from paper_2508_15532_b300 import workloads as W
from helpers import rel_err, run_gpu, run_oracle
from test_gpu_parity import small_flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_g3_flat_static_fp64_fp32_bf16():
    cfg, f = small_flat(nx=(10, 6, 4), n_geo=8, index=91)
    assert f["I"].shape[1] == 642
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 3)
    out = run_gpu(cfg, f, dt, 3, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    assert rel_err(out["E"], ref["E"]).max() < 1e-11
    o32 = run_gpu(cfg, f, dt, 3, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4
    # BF16 storage: the input and the output of each of the 6 stages round to
    # 2^-9 relative; the limited transport at most doubles an error it carries
    o16 = run_gpu(cfg, f, dt, 3, "bf16")
    assert rel_err(o16["I"], ref["I"], 1e-3).max() < 2 * (1 + 2 * 3) * 2.0 ** -9


def test_g3_flat_moving_fluid():
    cfg, f = small_flat(nx=(9, 6, 4), n_geo=8, index=92)
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + 192))
    v = rng.uniform(-0.3, 0.3, (len(f["rho"]), 3))
    gam = 1.0 / np.sqrt(1.0 - (v * v).sum(1))
    f["ucon"] = np.concatenate([gam[:, None], gam[:, None] * v], axis=1)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 2)
    out = run_gpu(cfg, f, dt, 2, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    assert np.abs(out["G"] - ref["G"]).max() < 1e-9 * np.abs(ref["G"]).max()
    o32 = run_gpu(cfg, f, dt, 2, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4


def test_g3_kerr_fp64():
    """The torus workload's recipe on a 12 x 16 x 4 Kerr-Schild box with pole
    boundaries and four pole-zeroed rows at each pole: geometry tables, n_0
    masks, the minimum-angle reconstruction and the angular edge fluxes at
    642 directions (rings of 5 and 6)."""
    cfg, f = W.kerr(nr=12, nth=16, nph=4, n_geo=8, index=93)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 2)
    assert (ref["E"] > 0).sum() > 100 and np.abs(ref["R"][:, 1:4]).max() > 0   # the torus is in the box
    out = run_gpu(cfg, f, dt, 2, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    assert rel_err(out["R"], ref["R"], 1e-6).max() < 1e-10
    # FP32 storage: E-bar and the flux moments at the spec bars (per
    # intensity the minimum-angle plane choice can flip, see
    # test_gpu_curvilinear.py)
    o32 = run_gpu(cfg, f, dt, 2, "fp32")
    assert o32["fails"] == 0
    assert rel_err(o32["E"], ref["E"], 1e-3).max() < 2e-5
    F, F32 = ref["R"][:, 1:4], o32["R"][:, 1:4]
    assert np.abs(F32 - F).max() < 1e-4 * np.abs(F).max()


def test_g3_cylindrical_tetrad_uniform_field():
    """A uniform isotropic field under the cylindrical tetrad (section 4.5):
    the CUDA path equals the oracle at 642 directions, and its one-step
    departure from uniformity (angular truncation) is smaller than at 162."""
    res = []
    for n_geo in (4, 8):
        cfg, f, dt, n, _ = CC.cylinder(N=(16, 16), n_geo=n_geo)
        cfg = dict(cfg, order=1)
        nd = 10 * n_geo * n_geo + 2
        f = dict(f, I=np.ones((16 * 16, nd)))
        dt1 = oracle.Oracle(cfg).cfl_dt(0.1)
        out = run_gpu(cfg, f, dt1, 1, "fp64")
        if n_geo == 8:
            ref = run_oracle(cfg, f, dt1, 1)
            assert rel_err(out["I"], ref["I"]).max() < 1e-11
        R = np.abs(out["I"] - 1.0).reshape(16, 16, nd)[2:-2, 2:-2] / dt1
        res.append(R.mean())
    assert res[1] < res[0] < 6e-3


def test_g3_spherical_front():
    """Section 4.1 on its own grid G3: the oracle and the CUDA path agree on a
    12^3 box, and on the 24^3 box the CUDA path's energy-weighted mean
    radius is within half a cell of t = 0.6 (FP64 and FP32)."""
    cfg, f, dt, n, x = CF.expansion(N=12, n_geo=8, t_end=0.3)
    ref = run_oracle(cfg, f, dt, n)
    out = run_gpu(cfg, f, dt, n, "fp64")
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    o32 = run_gpu(cfg, f, dt, n, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4
    cfg, f, dt, n, x = CF.expansion(N=24, n_geo=8, t_end=0.6)
    w = oracle.Oracle(dict(cfg, nx=(2, 2, 2))).grid()["w"]
    for prec in ("fp64", "fp32"):
        out = run_gpu(cfg, f, dt, n, prec)
        assert abs(CF.mean_radius(out["I"] @ w, x) - 0.6) < 0.5 * cfg["dx"][0], prec



@pytest.mark.parametrize("bc,limiter", [((("periodic", "periodic"),) * 3, "mc"),
                                        ((("outflow", "outflow"), ("periodic", "periodic"), ("periodic", "periodic")), "minmod")])
def test_g3_adjoint_against_oracle(bc, limiter):
    """The reverse pass at 642 directions (one CTA of 672 FP64 or 352 FP32
    threads per SM, 1 x 1 bricks) against the oracle adjoint, two steps on a
    9 x 4 x 4 box: FP64 within 1e-9 (floor 1e-6 of the largest component); the
    mixed pass (FP32 storage) as in test_gpu_adjoint.py: every component of
    the I0, kappa and eta gradients within MIXED_TOL of the largest component
    of its gradient (these seeded inputs put no limiter kink between the FP32
    and the FP64 forward states)."""
    from test_gpu_adjoint import MIXED_TOL, _gpu_adjoint, _loss_cotangents
    nx = (9, 4, 4)
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + 195))
    nc = int(np.prod(nx))
    cfg = W.base_config(8, nx, (0, 0, 0), tuple(1.0 / n for n in nx), bc, limiter=limiter)
    nd = 642
    rho = np.exp(rng.normal(0.0, 0.5, nc))
    T = rng.uniform(0.5, 2.0, nc)
    f = dict(rho=rho, ug=rho * T / (W.GAMMA - 1.0), ucon=W.static_ucon(nc),
             kappa=np.full(nc, 1e-2) * rng.uniform(0.5, 2.0, nc), alpha_s=np.full(nc, 0.4),
             eta=rng.uniform(0.5, 1.5, nc), I=W.planck(T)[:, None] * (1.0 + 0.1 * rng.uniform(-1, 1, (nc, nd))))
    nsteps = 2
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    dt = o.cfl_dt(0.4)
    w = o.grid()["w"]
    for precision in ("fp64", "fp32"):
        I0 = f["I"] if precision == "fp64" else np.asarray(f["I"], dtype=np.float32).astype(np.float64)
        o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
        o.set_intensity(I0)
        o.step(dt, nsteps)
        dI, du = _loss_cotangents(o.intensity(), o.ug(), w)
        o2 = oracle.Oracle(cfg)
        o2.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
        gI, gk, ge = o2.adjoint(I0, f["ug"], nsteps, dt, dI, du)
        Ib, ub, kb, eb = _gpu_adjoint(cfg, f, I0, dt, nsteps, dI, du, precision)
        if precision == "fp64":
            for name, got, ref in (("I0", Ib, gI), ("kappa", kb, gk), ("eta", eb, ge)):
                assert rel_err(got, ref, 1e-6).max() <= 1e-9, (name, rel_err(got, ref, 1e-6).max())
        else:
            for name, got, ref in (("I0", Ib, gI), ("kappa", kb, gk), ("eta", eb, ge)):
                err = np.abs(got - ref).max() / np.abs(ref).max()
                assert err <= MIXED_TOL, (name, err)
