"""Curved-space angular transport cases shared by the oracle pins and the GPU
parity tests: each returns (cfg, fields, dt, nsteps) for a vacuum run, with
the fields in the form tests/helpers.run_oracle and run_gpu take.

* tolman: I = (-n_0)^-4, an exact stationary vacuum solution of any
  stationary metric (I / nu^4 is constant along rays, nu proportional to
  1 / (-n_0)), on an axisymmetric (ln r, theta) patch of Kerr-Schild; with
  M = 0 it is the uniform field of flat space under the rotating spherical
  tetrad (section 4.5).
* orbit_bump: one equatorial cell near the prograde circular photon orbit of
  section 4.7, intensity concentrated around the direction of the photon
  that moves along phi only; the angular drift turns it inward inside the
  orbit and outward outside it.
* beam: a packet launched along phi-hat in flat spherical coordinates, which
  must travel on the straight line (section 4.5).
"""
import math

import numpy as np

import oracle
from paper_2508_15532_b300 import workloads as W


def vacuum_fields(nc, I):
    return dict(rho=np.zeros(nc), ug=np.zeros(nc), ucon=W.static_ucon(nc), kappa=np.zeros(nc),
                alpha_s=np.zeros(nc), eta=np.ones(nc), I=I)


def tolman(n_geo=4, a=0.9, M=1.0, r0=6.0, r1=7.0, t0=1.0, t1=1.2, N=16, order=1, cfl=0.1, nsteps=1):
    dx = ((math.log(r1) - math.log(r0)) / N, (t1 - t0) / N, 0.1)
    cfg = W.base_config(n_geo, (N, N, 1), (math.log(r0), t0, 0.0), dx,
                        (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                        coords="kerr_schild", a=a, M=M, order=order, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg)
    d = o.grid()["dir"]
    I = np.zeros((N * N, o.nd))
    for j in range(N):
        for i in range(N):
            x = [math.log(r0) + (i + 0.5) * dx[0], t0 + (j + 0.5) * dx[1], 0.05]
            g, e, _, _ = o.geometry_at(x)
            n0 = (e[0][None, :] + d @ e[1:]) @ g[:, 0]
            I[j * N + i] = (-n0) ** -4.0
    return cfg, vacuum_fields(N * N, I), o.cfl_dt(cfl), nsteps


def photon_orbit_radius(a):
    """Prograde circular photon orbit of Kerr (Bardeen, Press & Teukolsky 1972)."""
    return 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(-a)))


def orbit_bump(r, a=0.5, n_geo=4, width=0.05, dt=0.02, nsteps=25, mutant=0):
    """One cell at (r, pi/2); returns (cfg, fields, dt, nsteps, v_r) where v_r[s]
    is the coordinate radial speed d ln r / dt of grid direction s at the cell
    centre, from the oracle's tetrad."""
    dxl = 0.02
    cfg = W.base_config(n_geo, (1, 1, 1), (math.log(r) - dxl / 2, math.pi / 2 - dxl / 2, 0.0), (dxl, dxl, 0.1),
                        (("periodic",) * 2,) * 3, coords="kerr_schild", a=a, M=1.0, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg, mutant=mutant)
    g, e, _, _ = o.geometry_at([math.log(r), math.pi / 2, 0.05])
    # coordinate null vector with d ln r = d theta = 0: N = (1, 0, 0, Omega)
    A_, B_, C_ = g[3, 3], 2 * g[0, 3], g[0, 0]
    Om = (-B_ + math.sqrt(B_ * B_ - 4 * A_ * C_)) / (2 * A_)
    Na = np.linalg.solve(e.T, np.array([1.0, 0.0, 0.0, Om]))   # tetrad components: N = sum_a N^a e_a
    m0 = Na[1:] / Na[0]
    d = o.grid()["dir"]
    N = e[0][None, :] + d @ e[1:]
    v_r = N[:, 1] / N[:, 0]
    I = np.exp(-((d - m0) ** 2).sum(1) / width)[None, :]
    return cfg, vacuum_fields(1, I), dt, nsteps, v_r


def mean_vr(I, w, v_r):
    I = np.asarray(I).reshape(-1)
    return float((I * w * v_r).sum() / (I * w).sum())


def beam(N=16, n_geo=4, r0=1.5, ph0=0.3, T=0.8):
    """Equatorial wedge (ln r, phi) with one theta cell, flat space.  Returns
    (cfg, fields, dt, nsteps, centroid_error) where centroid_error(I) is the
    distance of the energy centroid of the final intensities from the straight
    line's point r0 r-hat + T phi-hat."""
    rlo, rhi, plo, phi_ = 1.0, 3.0, 0.0, 1.2
    dx = ((math.log(rhi) - math.log(rlo)) / N, 0.02, (phi_ - plo) / N)
    cfg = W.base_config(n_geo, (N, 1, N), (math.log(rlo), math.pi / 2 - 0.01, plo), dx,
                        (("outflow", "outflow"), ("periodic", "periodic"), ("outflow", "outflow")),
                        coords="kerr_schild", a=0.0, M=0.0, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg)
    g = o.grid()
    s_star = int(np.argmax(g["dir"] @ np.array([0.0, 0.0, 1.0])))
    rc = np.exp(math.log(rlo) + (np.arange(N) + 0.5) * dx[0])
    pc = plo + (np.arange(N) + 0.5) * dx[2]
    X = rc[None, :] * np.cos(pc)[:, None]
    Y = rc[None, :] * np.sin(pc)[:, None]
    I = np.zeros((N * N, o.nd))
    I[:, s_star] = np.exp(-((X - r0 * math.cos(ph0)) ** 2 + (Y - r0 * math.sin(ph0)) ** 2) / (2 * 0.05 ** 2)).ravel()
    n = int(math.ceil(T / o.cfl_dt(0.4)))
    w = g["w"]

    def centroid_error(J):
        E = (np.asarray(J) @ w).reshape(N, N) * (rc ** 3)[None, :]
        xc, yc = (E * X).sum() / E.sum(), (E * Y).sum() / E.sum()
        xe, ye = r0 * math.cos(ph0) - T * math.sin(ph0), r0 * math.sin(ph0) + T * math.cos(ph0)
        return math.hypot(xc - xe, yc - ye)

    return cfg, vacuum_fields(N * N, I), T / n, n, centroid_error
