"""The curved-space angular transport on the CUDA path (general stage kernel,
through the C ABI) against the FP64 oracle on the cases that pin the oracle's
angular drift, upwind side and pole map (tests/test_oracle_angular.py): the
stationary fields of Kerr-Schild and of flat spherical coordinates, the
donor-cell bump, the tangential beam and the photon-orbit bump of section
4.7, and the Kerr torus at 162 directions with pole boundaries.  FP64:
<= 1e-11 per intensity (floor 1e-6 of the largest); FP32 storage: <= 1e-4
(floor 1e-3).  Each case also checks on the GPU's own output the property
its oracle pin asserts."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle
from paper_2508_15532_b300 import workloads as W
import angular_cases as AC
from helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def both(cfg, f, dt, n, precisions=("fp64",)):
    ref = run_oracle(cfg, f, dt, n)
    outs = {}
    for p in precisions:
        out = run_gpu(cfg, f, dt, n, p)
        assert out["fails"] == 0
        bar, floor = (1e-11, 1e-6) if p == "fp64" else (1e-4, 1e-3)
        err = rel_err(out["I"], ref["I"], floor).max()
        assert err < bar, (p, err)
        outs[p] = out
    return ref, outs


@pytest.mark.parametrize("M,a,order", [(1.0, 0.9, 1), (1.0, 0.9, 2), (0.0, 0.0, 2)])
def test_stationary_fields(M, a, order):
    """I = (-n_0)^-4 (Kerr a = 0.9) and the uniform field of flat spherical
    coordinates (M = 0), three steps: parity, and the GPU's own residual
    |dI/dt| / I at the truncation level the oracle pin measures."""
    kw = dict(r0=2.0, r1=3.0, t0=0.7, t1=1.0) if M == 0.0 else {}
    cfg, f, dt, n = AC.tolman(n_geo=4, a=a, M=M, order=order, nsteps=3, **kw)
    ref, outs = both(cfg, f, dt, n, ("fp64", "fp32"))
    N = cfg["nx"][0]
    R = np.abs((outs["fp64"]["I"] - f["I"]) / (n * dt) / f["I"]).reshape(N, N, -1)[2:N - 2, 2:N - 2]
    assert R.mean() < 8e-3


def test_donor_bump_stays_non_negative():
    """Donor-cell angular transport (one flat spherical cell) for 50 steps:
    parity, no negative intensity, and the mean radial cosine grows."""
    cfg = W.base_config(4, (1, 1, 1), (math.log(3.0), 1.1, 0.0), (0.05, 0.05, 0.05), (("periodic",) * 2,) * 3,
                        coords="kerr_schild", a=0.0, M=0.0, source=False, n0_cut=0.0, order=1, ang_recon="donor")
    o = oracle.Oracle(cfg)
    g = o.grid()
    d, w = g["dir"], g["w"]
    c = np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])
    I = np.exp(-((d - c) ** 2).sum(1) / 0.05)[None, :]
    ref, outs = both(cfg, AC.vacuum_fields(1, I), 0.05, 50, ("fp64", "fp32"))
    for out in outs.values():
        J = out["I"][0]
        assert J.min() >= -1e-15
        assert (J * w * d[:, 0]).sum() / (J * w).sum() > (I[0] * w * d[:, 0]).sum() / (I[0] * w).sum() + 0.2


def test_tangential_beam_straight():
    """Section 4.5: a packet launched along phi-hat in flat spherical
    coordinates stays within two cells of the straight line."""
    cfg, f, dt, n, cerr = AC.beam()
    ref, outs = both(cfg, f, dt, n)
    assert cerr(outs["fp64"]["I"]) < 0.15


@pytest.mark.parametrize("n_geo", [4, 8])
def test_photon_orbit_bump_turns(n_geo):
    """Section 4.7: the tangential photon's direction bump turns inward just
    inside the prograde photon orbit of a = 0.5 and outward just outside it
    (162 directions, and the section's own 642).  At 642 directions the bump
    spans more near-tied reconstruction planes, and FP32 rounding flips some
    of them (the minimum-angle choice is discontinuous; see
    test_gpu_curvilinear.py): measured 2.5e-4 per intensity, held to that
    file's 5e-2 flip bar; the turn itself is checked on the FP64 run."""
    r1 = AC.photon_orbit_radius(0.5)
    turn = {}
    for fr in (0.95, 1.0, 1.05):
        cfg, f, dt, n, vr = AC.orbit_bump(fr * r1, n_geo=n_geo)
        ref, outs = both(cfg, f, dt, n, ("fp64", "fp32") if n_geo == 4 else ("fp64",))
        if n_geo != 4:
            o32 = run_gpu(cfg, f, dt, n, "fp32")
            assert rel_err(o32["I"], ref["I"], 1e-3).max() < 5e-2
        w = oracle.Oracle(cfg).grid()["w"]
        turn[fr] = AC.mean_vr(outs["fp64"]["I"], w, vr) - AC.mean_vr(f["I"], w, vr)
    assert turn[0.95] - turn[1.0] < -2e-4
    assert turn[1.05] - turn[1.0] > 2e-4


@pytest.mark.parametrize("nph", [1, 8])
def test_kerr_torus_162_directions_fp64(nph):
    """The Kerr torus (a = 0.9) at the workloads' 162 directions, with pole
    boundaries and pole zeroing, minimum-angle reconstruction and the boosted
    interaction: FP64 parity over 3 steps."""
    cfg, f = W.kerr(nr=24, nth=16, nph=nph, n_geo=4, index=51 + nph)
    dt = oracle.Oracle(cfg).cfl_dt(0.4)
    ref = run_oracle(cfg, f, dt, 3)
    out = run_gpu(cfg, f, dt, 3, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    assert rel_err(out["ug"], ref["ug"]).max() < 1e-11
    assert rel_err(out["R"], ref["R"], 1e-6).max() < 1e-10
