"""The oracle's hand-derived reverse mode against central finite differences
of its own forward rollout (section 5.2: gradients of a loss over a
differentiable rollout; section 3.5.2 for the interaction being reversed).

Finite differences are an independent pin: they use only the forward step,
which is pinned separately.  A relative step of 1e-4 leaves truncation and
rounding errors near 1e-6, so agreement to 1e-5 of the largest gradient
component checks every term of the reverse pass.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15532_b300 import workloads as W

HREL = 1e-4
TOL = 1e-5


def _setup(order=2, limiter=None, index=50, N=6, transport=True):
    cfg, f = W.flat3d(N=N, n_geo=2, index=index)
    cfg = dict(cfg)
    cfg["order"] = order
    cfg["transport"] = transport
    if limiter is not None:
        cfg["limiter"] = limiter
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    return cfg, f, o


def _loss(cfg, f, dt, nsteps, w, kappa, eta, I0, ug0):
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], ug0, f["ucon"], kappa, f["alpha_s"], eta)
    o.set_intensity(I0)
    o.step(dt, nsteps)
    E = o.intensity() @ w
    ug = o.ug()
    # a loss that couples the radiation energy and the gas energy
    return float((E ** 2).sum() + 3.0 * (ug * E).sum()), o.intensity(), E, ug


@pytest.mark.parametrize("order,limiter,transport", [(2, None, True), (1, None, True), (2, "minmod", True),
                                                     (2, None, False), (1, None, False)])
def test_adjoint_matches_finite_differences(order, limiter, transport):
    """transport False: a source-only configuration, where each stage of
    section 3.6 leaves its base unchanged and only the interaction acts"""
    cfg, f, o = _setup(order=order, limiter=limiter, transport=transport)
    nsteps = 3
    dt = o.cfl_dt(0.4)
    w = o.grid()["w"]
    L0, IN, EN, ugN = _loss(cfg, f, dt, nsteps, w, f["kappa"], f["eta"], f["I"], f["ug"])
    dLdI = (2.0 * EN + 3.0 * ugN)[:, None] * w[None, :]
    dLdug = 3.0 * EN
    gI, gk, ge = o.adjoint(f["I"], f["ug"], nsteps, dt, dLdI, dLdug)
    scale = {"kappa": np.abs(gk).max(), "eta": np.abs(ge).max(), "I0": np.abs(gI).max()}
    rng = np.random.default_rng(7 + order)
    cells = rng.choice(len(EN), 5, replace=False)
    for c in cells:
        for name, grad in (("kappa", gk), ("eta", ge)):
            base = f[name]
            h = HREL * base[c]
            a1 = base.copy(); a1[c] += h
            a2 = base.copy(); a2[c] -= h
            k1, e1 = (a1, f["eta"]) if name == "kappa" else (f["kappa"], a1)
            k2, e2 = (a2, f["eta"]) if name == "kappa" else (f["kappa"], a2)
            fd = (_loss(cfg, f, dt, nsteps, w, k1, e1, f["I"], f["ug"])[0]
                  - _loss(cfg, f, dt, nsteps, w, k2, e2, f["I"], f["ug"])[0]) / (2 * h)
            assert abs(grad[c] - fd) <= TOL * max(abs(fd), scale[name]), (name, c, grad[c], fd)
        s = int(rng.integers(0, o.nd))
        h = HREL * f["I"][c, s]
        I1 = f["I"].copy(); I1[c, s] += h
        I2 = f["I"].copy(); I2[c, s] -= h
        fd = (_loss(cfg, f, dt, nsteps, w, f["kappa"], f["eta"], I1, f["ug"])[0]
              - _loss(cfg, f, dt, nsteps, w, f["kappa"], f["eta"], I2, f["ug"])[0]) / (2 * h)
        assert abs(gI[c, s] - fd) <= TOL * max(abs(fd), scale["I0"]), ("I0", c, s, gI[c, s], fd)


def test_adjoint_linear_in_cotangent():
    """The reverse pass is linear in the cotangent it is seeded with."""
    cfg, f, o = _setup(order=2)
    dt = o.cfl_dt(0.4)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((o.ncell, o.nd)); b = rng.standard_normal((o.ncell, o.nd))
    ua = rng.standard_normal(o.ncell); ub = rng.standard_normal(o.ncell)
    ga = o.adjoint(f["I"], f["ug"], 2, dt, a, ua)
    gb = o.adjoint(f["I"], f["ug"], 2, dt, b, ub)
    gab = o.adjoint(f["I"], f["ug"], 2, dt, 2.0 * a - b, 2.0 * ua - ub)
    for x, y, z in zip(ga, gb, gab):
        np.testing.assert_allclose(z, 2.0 * x - y, rtol=1e-9, atol=1e-12 * np.abs(z).max())


def test_adjoint_rejects_moving_fluid():
    cfg, f = W.flat3d(N=4, n_geo=2, index=51)
    o = oracle.Oracle(dict(cfg))
    ucon = f["ucon"].copy()
    ucon[:, 1] = 0.1
    ucon[:, 0] = np.sqrt(1.0 + 0.01)
    o.set_fluid(f["rho"], f["ug"], ucon, f["kappa"], f["alpha_s"], f["eta"])
    with pytest.raises(RuntimeError, match="rest"):
        o.adjoint(f["I"], f["ug"], 1, 1e-3, np.zeros((o.ncell, o.nd)), np.zeros(o.ncell))
