"""Flat space under a rotating tetrad (sections 4.5 and 4.6), shared by the
oracle pins and the GPU parity tests: a packet launched in one grid
direction must travel on a straight line in Cartesian space, although its
direction in the tetrad frame turns as it moves (the angular fluxes carry
it from one grid direction to the next).

* snake(): snake coordinates (w, y, z), w = x - A sin(k pi y) (App. A.1,
  A = 0.1, k = 2 as in section 4.6), Gram-Schmidt tetrad: the frame turns
  with y by atan(A k pi cos(k pi y));
* cylinder(): Cartesian coordinates with the tetrad aligned with the
  cylindrical unit vectors (section 4.5): the frame turns with atan2(y, x).
Each returns (cfg, fields, dt, nsteps, centroid_error), centroid_error(I)
being the distance between the packet's Cartesian energy centroid and the
straight line's point after the run."""
import math

import numpy as np

import oracle
from paper_2508_15532_b300 import workloads as W


def _vacuum(nc, nd):
    return dict(rho=np.zeros(nc), ug=np.zeros(nc), ucon=W.static_ucon(nc), kappa=np.zeros(nc),
                alpha_s=np.zeros(nc), eta=np.ones(nc), I=np.zeros((nc, nd)))


def _launch(o, x_logical, target_cart, to_cart_vec):
    """Grid direction nearest the Cartesian direction target_cart at the
    logical point x_logical, and that direction's exact Cartesian velocity
    there.  to_cart_vec maps a coordinate 4-vector to Cartesian components."""
    g, e, _, _ = o.geometry_at(list(x_logical))
    d = o.grid()["dir"]
    best, vbest = -2.0, None
    for s in range(o.nd):
        N = e[0] + d[s] @ e[1:]                  # coordinate components of (1, n-hat)
        v = to_cart_vec(N)
        v = v[1:3] / v[0]
        if np.linalg.norm(v) < 1e-9:            # a direction along z
            continue
        c = float(v @ target_cart) / np.linalg.norm(v)
        if c > best:
            best, sbest, vbest = c, s, v
    return sbest, vbest


def snake(N=(64, 32), n_geo=4, A=0.1, k=2.0, start=(0.5, 0.2), psi=45.0, t_end=0.5):
    nw, ny = N
    dx = (2.0 / nw, 1.0 / ny, 0.1)
    cfg = W.base_config(n_geo, (nw, ny, 1), (0.0, 0.0, 0.0), dx,
                        (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                        coords="snake", snake_A=A, snake_k=k, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg)
    wc = (np.arange(nw) + 0.5) * dx[0]
    yc = (np.arange(ny) + 0.5) * dx[1]
    Y, Wc = np.meshgrid(yc, wc, indexing="ij")
    X = Wc + A * np.sin(k * math.pi * Y)          # Cartesian x of the cell centres
    xs, ys = start
    ws = xs - A * math.sin(k * math.pi * ys)

    def to_cart(Nv):                              # (t, w, y, z) -> (t, x, y)
        delta = A * k * math.pi * math.cos(k * math.pi * ys)
        return np.array([Nv[0], Nv[1] + delta * Nv[2], Nv[2]])

    s, v = _launch(o, (ws, ys, 0.05), np.array([math.cos(math.radians(psi)), math.sin(math.radians(psi))]), to_cart)
    f = _vacuum(nw * ny, o.nd)
    f["I"][:, s] = np.exp(-((X - xs) ** 2 + (Y - ys) ** 2) / (2 * 0.04 ** 2)).ravel()
    n = int(math.ceil(t_end / o.cfl_dt(0.4)))
    w = o.grid()["w"]

    def centroid_error(I):
        E = np.asarray(I) @ w                     # sqrt(-g) = 1: equal cell volumes
        c = np.array([(E * X.ravel()).sum(), (E * Y.ravel()).sum()]) / E.sum()
        return float(np.linalg.norm(c - (np.array(start) + v * t_end)))

    return cfg, f, t_end / n, n, centroid_error


def cylinder(N=(48, 48), n_geo=4, start=(1.4, -0.6), psi=60.0, t_end=0.8):
    nx, ny = N
    lo = (1.0, -1.0)
    dx = (2.0 / nx, 2.0 / ny, 0.1)
    cfg = W.base_config(n_geo, (nx, ny, 1), (lo[0], lo[1], 0.0), dx,
                        (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                        coords="cart_cyl_tetrad", source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg)
    xc = lo[0] + (np.arange(nx) + 0.5) * dx[0]
    yc = lo[1] + (np.arange(ny) + 0.5) * dx[1]
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    s, v = _launch(o, (start[0], start[1], 0.05),
                   np.array([math.cos(math.radians(psi)), math.sin(math.radians(psi))]), lambda Nv: Nv[:3])
    f = _vacuum(nx * ny, o.nd)
    f["I"][:, s] = np.exp(-((X - start[0]) ** 2 + (Y - start[1]) ** 2) / (2 * 0.05 ** 2)).ravel()
    n = int(math.ceil(t_end / o.cfl_dt(0.4)))
    w = o.grid()["w"]

    def centroid_error(I):
        E = np.asarray(I) @ w
        c = np.array([(E * X.ravel()).sum(), (E * Y.ravel()).sum()]) / E.sum()
        return float(np.linalg.norm(c - (np.array(start) + v * t_end)))

    return cfg, f, t_end / n, n, centroid_error
