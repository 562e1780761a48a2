"""The flat-space transport tests of section 4 with closed-form behaviour on
the CUDA path, against the FP64 oracle (<= 1e-11 per intensity, floor 1e-6
of the largest) and against the closed-form property each case pins on the
oracle (tests/test_oracle_closed_forms.py): the spherical light front at
r = ct, the 1/d^2 flux of a steady source, and crossing beams that pass
through each other unperturbed.  FP32 storage is held to 1e-4 (floor 1e-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle
import closed_form_cases as CF
from helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def both(cfg, f, dt, n):
    ref = run_oracle(cfg, f, dt, n)
    out = run_gpu(cfg, f, dt, n, "fp64")
    assert out["fails"] == 0
    assert rel_err(out["I"], ref["I"]).max() < 1e-11
    o32 = run_gpu(cfg, f, dt, n, "fp32")
    assert rel_err(o32["I"], ref["I"], 1e-3).max() < 1e-4
    return ref, out


def test_spherical_front_gpu():
    cfg, f, dt, n, x = CF.expansion(t_end=0.6)
    ref, out = both(cfg, f, dt, n)
    w = oracle.Oracle(cfg).grid()["w"]
    assert abs(CF.mean_radius(out["I"] @ w, x) - 0.6) < 0.5 * cfg["dx"][0]


def test_inverse_square_gpu():
    cfg, f, dt, n, x = CF.inverse_square()
    ref, out = both(cfg, f, dt, n)
    F = out["R"][:, 1:4]
    rr = np.linalg.norm(x, axis=1)
    Fr = (F * x).sum(1) / np.maximum(rr, 1e-12)
    radii = np.array([0.4, 0.5, 0.6, 0.7, 0.8])
    Fd2 = CF.shell_means(Fr, x, radii, 0.1) * radii ** 2
    assert Fd2.max() / Fd2.min() < 1.03, Fd2


def test_colliding_beams_gpu():
    runs = {}
    for which in ((True, True), (True, False), (False, True)):
        cfg, f, dt, n, x, (s1, s2), d, starts = CF.colliding_packets(which=which)
        if which == (True, True):
            ref, out = both(cfg, f, dt, n)
            runs[which] = out["I"]
        else:
            runs[which] = run_gpu(cfg, f, dt, n, "fp64")["I"]
    assert np.array_equal(runs[(True, True)], runs[(True, False)] + runs[(False, True)])
    for s, c0 in ((s1, starts[0]), (s2, starts[1])):
        c = CF.centroid(runs[(True, True)][:, s], x)
        assert np.linalg.norm(c - (np.array(c0) + d[s] * dt * n)) < 0.1 * cfg["dx"][0]
