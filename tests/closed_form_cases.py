"""Flat-space transport cases of section 4 with closed-form truth, shared by
the oracle pins (test_oracle_closed_forms.py) and the GPU parity tests
(test_gpu_closed_forms.py).  Each returns (cfg, fields, dt, nsteps) plus what
its check needs; fields are in the form tests/helpers.run_oracle takes.

* expansion (section 4.1): an isotropic source of about 3 cells at the centre
  of a vacuum box; its light front moves out at c, so the energy-weighted mean
  radius of the radiation grows as r(t) = t once t is large next to the source.
* inverse_square (section 4.2): a hot, optically thick sphere whose gas holds
  far more energy than it radiates (so its temperature stays put) shines into
  vacuum; in the steady state the flux through every shell is the luminosity,
  and the free-streaming energy density averaged over a shell falls as 1/d^2.
* colliding_beams (section 4.3): two packets crossing each other in vacuum
  pass through unperturbed: in flat Cartesian geometry without matter every
  direction evolves on its own, so the run with both packets equals, direction
  by direction, the runs with one packet each.
"""
import math

import numpy as np

from paper_2508_15532_b300 import workloads as W


def _box(N, n_geo, half=1.0, **kw):
    dx = 2.0 * half / N
    cfg = W.base_config(n_geo, (N, N, N), (-half, -half, -half), (dx, dx, dx),
                        (("outflow", "outflow"),) * 3, **kw)
    c = -half + (np.arange(N) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return cfg, np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), dx


def vacuum(nc, nd):
    return dict(rho=np.zeros(nc), ug=np.zeros(nc), ucon=W.static_ucon(nc), kappa=np.zeros(nc),
                alpha_s=np.zeros(nc), eta=np.ones(nc), I=np.zeros((nc, nd)))


def expansion(N=24, n_geo=2, t_end=0.6, source_radius=None):
    """Returns (cfg, fields, dt, nsteps, x): x the cell centres [nc, 3]."""
    cfg, x, dx = _box(N, n_geo, source=False)
    nd = 10 * n_geo * n_geo + 2
    f = vacuum(N ** 3, nd)
    r = np.linalg.norm(x, axis=1)
    src = r < (1.6 * dx if source_radius is None else source_radius)
    f["I"][src] = 1.0
    dt0 = 0.4 * dx          # the bound of section 3.7 for |n^a| <= 1 (slightly below it)
    n = int(math.ceil(t_end / dt0))
    return cfg, f, t_end / n, n, x


def mean_radius(E, x):
    r = np.linalg.norm(x, axis=1)
    return float((E * r).sum() / E.sum())


def inverse_square(N=24, n_geo=2, t_end=2.0, R=0.2, T=1.0):
    """Returns (cfg, fields, dt, nsteps, x)."""
    cfg, x, dx = _box(N, n_geo, rho_exp=1.0, T_exp=0.0)
    nd = 10 * n_geo * n_geo + 2
    nc = N ** 3
    f = vacuum(nc, nd)
    r = np.linalg.norm(x, axis=1)
    hot = r < R
    rho = np.where(hot, 1.0e4, 0.0)
    f.update(rho=rho, ug=rho * T / (W.GAMMA - 1.0), kappa=np.where(hot, 2.0e-3 / dx, 0.0))   # tau ~ 20 per cell
    f["I"][hot] = W.planck(T)
    dt0 = 0.4 * dx
    n = int(math.ceil(t_end / dt0))
    return cfg, f, t_end / n, n, x


def shell_means(E, x, radii, width):
    """Energy density averaged over the cells of each shell |r - d| < width/2."""
    r = np.linalg.norm(x, axis=1)
    return np.array([E[np.abs(r - d) < width / 2].mean() for d in radii])


def colliding_packets(N=24, n_geo=2, t_end=1.0, which=(True, True)):
    """Two Gaussian packets at (-0.5, 0, -0.3) and (0.5, 0, -0.3) launched
    along the grid directions nearest (cos 32 deg, 0, sin 32 deg) and
    (-cos 32 deg, 0, sin 32 deg) (icosahedron vertices of the n = 2 grid); they
    cross near the origin at t ~ 0.6, at an angle of about 64 degrees.
    Returns (cfg, fields, dt, nsteps, x, (s1, s2), dirs, starts)."""
    cfg, x, dx = _box(N, n_geo, source=False)
    import oracle
    d = oracle.Oracle(dict(cfg, nx=(2, 2, 2))).grid()["dir"]
    a = math.radians(32.0)
    s1 = int(np.argmax(d @ np.array([math.cos(a), 0.0, math.sin(a)])))
    s2 = int(np.argmax(d @ np.array([-math.cos(a), 0.0, math.sin(a)])))
    starts = ((-0.5, 0.0, -0.3), (0.5, 0.0, -0.3))
    nd = d.shape[0]
    f = vacuum(N ** 3, nd)
    for on, c0, s in ((which[0], starts[0], s1), (which[1], starts[1], s2)):
        if on:
            f["I"][:, s] += np.exp(-((x - np.array(c0)) ** 2).sum(1) / (2 * 0.1 ** 2))
    dt0 = 0.4 * dx
    n = int(math.ceil(t_end / dt0))
    return cfg, f, t_end / n, n, x, (s1, s2), d, starts


def centroid(e, x):
    return (e[:, None] * x).sum(0) / e.sum()
