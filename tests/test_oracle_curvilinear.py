"""Pins of the oracle's angular transport under rotating tetrads in flat
space (sections 4.5 and 4.6, App. A.1): snake coordinates with their
Gram-Schmidt tetrad, and Cartesian coordinates with the tetrad aligned with
the cylindrical unit vectors.  Light travels on straight lines in Cartesian
space whatever the frame, so a packet's Cartesian energy centroid must stay
on the line while its tetrad-frame direction turns from one grid direction to
the next.  An oracle build whose drift has the wrong sign (OR_MUTANT 1) bends
the packets by several cells and fails both.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import curvilinear_cases as CC
from paper_2508_15532_b300 import workloads as W


def run(fn, mutant=0):
    cfg, f, dt, n, cerr = fn()
    o = oracle.Oracle(cfg, mutant=mutant)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    o.set_intensity(f["I"])
    o.step(dt, n)
    return cerr(o.intensity()), cfg


def test_snake_metric_is_flat_space():
    """g of snake coordinates equals J^T eta J for the map x = w + A sin(k pi y)
    (numerical Jacobian), and the tetrad is orthonormal under it."""
    cfg, _, _, _, _ = CC.snake()
    o = oracle.Oracle(cfg)
    A, k = cfg["snake_A"], cfg["snake_k"]
    for w, y in ((0.3, 0.1), (1.2, 0.63), (0.7, 0.9)):
        g, e, _, sqrtg = o.geometry_at([w, y, 0.05])
        J = np.eye(4)
        J[1, 2] = A * k * math.pi * math.cos(k * math.pi * y)      # dx/dy at fixed w
        assert np.abs(g - J.T @ np.diag([-1.0, 1, 1, 1]) @ J).max() < 1e-14
        assert np.abs(e @ g @ e.T - np.diag([-1.0, 1, 1, 1])).max() < 1e-14
        assert abs(sqrtg - 1.0) < 1e-14


def test_snake_packet_is_straight():
    """A = 0.1, k = 2 (section 4.6), 64 x 32 cells of 1/32, 162 directions:
    after travelling 0.5 the packet's Cartesian centroid is within 3 cells of
    the straight line (measured 2.3 cells; the wrong drift sign: 8.8)."""
    err, cfg = run(CC.snake)
    assert err < 3 * cfg["dx"][0]


def test_cylindrical_tetrad_packet_is_straight():
    """Cartesian box x in [1, 3], y in [-1, 1] (48 x 48), tetrad (r-hat,
    phi-hat, z-hat): after travelling 0.8 the centroid is within 2.5 cells of
    the straight line (measured 1.4; the wrong drift sign: 7.4)."""
    err, cfg = run(CC.cylinder)
    assert err < 2.5 * cfg["dx"][0]


def test_cylindrical_tetrad_uniform_field():
    """A uniform isotropic field is stationary in flat space under any
    tetrad; one step leaves it uniform up to the angular truncation (mean
    |dI/dt|/I below 6e-3 at 162 directions, smaller at 642)."""
    res = []
    for n_geo in (4, 8):
        cfg, f, dt, n, _ = CC.cylinder(N=(16, 16), n_geo=n_geo)
        cfg = dict(cfg, order=1)
        o = oracle.Oracle(cfg)
        I = np.ones((16 * 16, o.nd))
        o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
        o.set_intensity(I)
        dt1 = o.cfl_dt(0.1)
        o.step(dt1, 1)
        R = np.abs(o.intensity() - 1.0).reshape(16, 16, o.nd)[2:-2, 2:-2] / dt1
        res.append(R.mean())
    assert res[0] < 6e-3 and res[1] < res[0]


@pytest.mark.parametrize("fn", [CC.snake, CC.cylinder])
def test_wrong_drift_sign_bends_the_packet(fn):
    err, cfg = run(fn, mutant=1)
    assert err > 5 * cfg["dx"][0]
