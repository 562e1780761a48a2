"""Pins of the oracle's curved-space angular transport and pole boundary
against what geometry fixes independently of the oracle's code:

* the tangent drift of every geodesic-grid edge equals the rate at which a
  photon's tetrad-frame direction turns along a geodesic integrated here from
  the textbook Kerr-Schild metric (eq. angular_n_vectors, eq. angular_fluxes);
* I = C (-n_0)^-4 is an exact stationary vacuum solution in any stationary
  metric (I / nu^4 is constant along rays and nu = -p_0 / (-n_0)), so one
  transport step leaves it unchanged up to truncation that shrinks with the
  angular resolution; in flat space with the spherical tetrad it is a uniform
  field (section 4.5's rotating-tetrad setting);
* the angular flux is upwind (eq. angular_fluxes): donor-cell angular transport
  keeps intensities non-negative;
* a beam launched tangentially in flat spherical coordinates follows the
  straight line (section 4.5);
* the pole ghost is the analytic continuation of the spherical chart through
  theta = 0 (theta -> -theta seen from phi + pi, theta-hat and phi-hat reversed).

Builds of the oracle with one planted mistake (oracle/build.py, OR_MUTANT)
fail at least one of these pins.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2508_15532_b300 import workloads as W
import angular_cases as AC

ETA = np.diag([-1.0, 1, 1, 1])


# --------------------------------------------------------------- independent geometry
def ks_metric(x, a, M):
    """Kerr-Schild metric in (t, ln r, theta, phi) from the textbook form eta + 2 H l l."""
    r, th = math.exp(x[0]), x[1]
    sig = r * r + a * a * math.cos(th) ** 2
    H, s2 = M * r / sig, math.sin(th) ** 2
    g = np.zeros((4, 4))
    g[0, 0] = -1; g[1, 1] = 1; g[1, 3] = g[3, 1] = -a * s2; g[2, 2] = sig; g[3, 3] = (r * r + a * a) * s2
    l = np.array([1.0, 1.0, 0.0, -a * s2])
    J = np.diag([1.0, r, 1.0, 1.0])
    return J @ (g + 2 * H * np.outer(l, l)) @ J


def christoffel(x, a, M, h=1e-5):
    g = ks_metric(x, a, M)
    gi = np.linalg.inv(g)
    dg = np.zeros((4, 4, 4))
    for mu in (1, 2):
        xp, xm = list(x), list(x)
        xp[mu - 1] += h; xm[mu - 1] -= h
        dg[mu] = (ks_metric(xp, a, M) - ks_metric(xm, a, M)) / (2 * h)
    return 0.5 * (np.einsum("bl,mln->bmn", gi, dg) + np.einsum("bl,nlm->bmn", gi, dg) - np.einsum("bl,lmn->bmn", gi, dg))


def one_cell_ks(r, th, a, M, n_geo=2, mutant=0, **kw):
    dx = (0.02, 0.02, 0.1)
    cfg = W.base_config(n_geo, (1, 1, 1), (math.log(r) - dx[0] / 2, th - dx[1] / 2, 0.0), dx,
                        (("periodic",) * 2,) * 3, coords="kerr_schild", a=a, M=M, **kw)
    return oracle.Oracle(cfg, mutant=mutant)


def geodesic_edge_speeds(o, x, a, M, h=1e-5):
    """n_0(m) (dm/dlambda . u_e) at every edge midpoint m, with dN/dlambda from
    the geodesic equation of the independent metric and the tetrad legs of the
    oracle (pinned separately: orthonormal under this metric, eq. tetrad_def)."""
    g, e, _, _ = o.geometry_at(x)
    gind = ks_metric(x, a, M)
    ei = ETA @ e @ gind
    Gam = christoffel(x, a, M)
    dei = np.zeros((4, 4, 4))
    for nu in (1, 2):
        xp, xm = list(x), list(x)
        xp[nu - 1] += h; xm[nu - 1] -= h
        gp, ep, _, _ = o.geometry_at(xp)
        gm, em, _, _ = o.geometry_at(xm)
        dei[nu] = (ETA @ ep @ ks_metric(xp, a, M) - ETA @ em @ ks_metric(xm, a, M)) / (2 * h)
    gr = o.grid()
    out = np.zeros(o.ne)
    for k in range(o.ne):
        m, u = gr["emid"][k], gr["eu"][k]
        N = e.T @ np.concatenate([[1.0], m])                 # coordinate N^mu of tetrad N^a = (1, m)
        dNc = -np.einsum("mab,a,b->m", Gam, N, N)            # geodesic equation
        dNa = np.einsum("nam,n,m->a", dei, N, N) + ei @ dNc  # tetrad components
        v = dNa[1:] - m * dNa[0]                             # turn rate of m = N^i / N^0
        out[k] = (gind[0] @ N) * (v @ u)
    return out


DRIFT_POINTS = [(0.9, 1.0, 3.0, 1.1), (0.9, 1.0, 7.0, 0.4), (0.0, 0.0, 2.5, 0.8),
                # just inside and outside the prograde circular photon orbit of a = 0.5 (section 4.7)
                (0.5, 1.0, 0.95 * 2.3473, math.pi / 2), (0.5, 1.0, 1.05 * 2.3473, math.pi / 2)]


def drift_error(a, M, r, th, mutant=0):
    o = one_cell_ks(r, th, a, M, mutant=mutant)
    w = o.edge_speeds(0)
    wg = geodesic_edge_speeds(o, [math.log(r), th, 0.05], a, M)
    return np.abs(w - wg).max() / np.abs(wg).max()


@pytest.mark.parametrize("a,M,r,th", DRIFT_POINTS)
def test_drift_is_the_geodesic_turn_rate(a, M, r, th):
    assert drift_error(a, M, r, th) < 1e-8


def photon_orbit_fate(a, r, dlam=2.0, n=4000):
    """Tangential prograde photon in the equatorial plane at radius r, traced by
    RK4 on the geodesic equation of the independent metric: +1 if it escapes
    outward, -1 if it falls in."""
    def rhs(y):
        x, N = y[:4], y[4:]
        return np.concatenate([N, -np.einsum("mab,a,b->m", christoffel(x[1:], a, 1.0), N, N)])
    g = ks_metric([math.log(r), math.pi / 2, 0.0], a, 1.0)
    # null vector with dr = dtheta = 0: N = (1, 0, 0, Omega), g_tt + 2 g_tphi O + g_phiphi O^2 = 0
    A_, B_, C_ = g[3, 3], 2 * g[0, 3], g[0, 0]
    Om = (-B_ + math.sqrt(B_ * B_ - 4 * A_ * C_)) / (2 * A_)
    y = np.array([0.0, math.log(r), math.pi / 2, 0.0, 1.0, 0.0, 0.0, Om])
    h = dlam / n
    for _ in range(n):
        k1 = rhs(y); k2 = rhs(y + 0.5 * h * k1); k3 = rhs(y + 0.5 * h * k2); k4 = rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return math.copysign(1.0, y[1] - math.log(r))


def test_photon_orbit_direction():
    """Section 4.7: radiation started tangentially just inside the prograde
    circular photon orbit falls in, just outside it escapes.  The geodesics
    traced here are the characteristics the oracle's drift follows (previous
    test, including these two radii)."""
    r1 = 2 * (1 + math.cos(2.0 / 3.0 * math.acos(-0.5)))
    assert photon_orbit_fate(0.5, 0.95 * r1) < 0
    assert photon_orbit_fate(0.5, 1.05 * r1) > 0


def orbit_turn(f, mutant=0, n_geo=4):
    """Change of the mean coordinate radial speed <d ln r/dt> of a direction bump
    started on the tangential photon at f r_1 (a = 0.5), minus the same change
    at r_1 itself (which removes the part due to the bump's spreading)."""
    r1 = AC.photon_orbit_radius(0.5)
    out = []
    for r in (f * r1, r1):
        cfg, fl, dt, n, vr = AC.orbit_bump(r, mutant=mutant, n_geo=n_geo)
        o = oracle.Oracle(cfg, mutant=mutant)
        o.set_fluid(fl["rho"], fl["ug"], fl["ucon"], fl["kappa"], fl["alpha_s"], fl["eta"])
        o.set_intensity(fl["I"])
        o.step(dt, n)
        w = o.grid()["w"]
        out.append(AC.mean_vr(o.intensity(), w, vr) - AC.mean_vr(fl["I"], w, vr))
    return out[0] - out[1]


def test_photon_orbit_drift_direction():
    """Section 4.7 as a directional pin of the oracle's angular drift: radiation
    moving tangentially just inside the prograde circular photon orbit turns
    inward (its mean radial speed falls), just outside it turns outward.
    Measured: -4.4e-4 at 0.95 r_1, +4.9e-4 at 1.05 r_1 after t = 0.5; a drift of
    the opposite sign gives +1.1e-3 and -8.6e-4.  On the section's own grid G3
    (642 directions): -7.3e-4 and +6.5e-4."""
    assert orbit_turn(0.95) < -2e-4
    assert orbit_turn(1.05) > 2e-4
    assert orbit_turn(0.95, n_geo=8) < -4e-4
    assert orbit_turn(1.05, n_geo=8) > 4e-4


# --------------------------------------------------------------- stationary fields
def tolman_residual(n_geo, a=0.9, M=1.0, r0=6.0, r1=7.0, t0=1.0, t1=1.2, N=16, mutant=0):
    """Mean and largest |dI/dt| / I over interior cells after one first-order
    transport step (vacuum) of I = (-n_0)^-4 on an axisymmetric (r, theta) patch."""
    dx = ((math.log(r1) - math.log(r0)) / N, (t1 - t0) / N, 0.1)
    cfg = W.base_config(n_geo, (N, N, 1), (math.log(r0), t0, 0.0), dx,
                        (("outflow", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                        coords="kerr_schild", a=a, M=M, order=1, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg, mutant=mutant)
    d = o.grid()["dir"]
    I = np.zeros((N * N, o.nd))
    for j in range(N):
        for i in range(N):
            x = [math.log(r0) + (i + 0.5) * dx[0], t0 + (j + 0.5) * dx[1], 0.05]
            g, e, _, _ = o.geometry_at(x)
            n0 = (e[0][None, :] + d @ e[1:]) @ g[:, 0]
            I[j * N + i] = (-n0) ** -4.0
    o.set_fluid(np.zeros(N * N), np.zeros(N * N), W.static_ucon(N * N), np.zeros(N * N), np.zeros(N * N))
    o.set_intensity(I)
    dt = o.cfl_dt(0.1)
    o.step(dt, 1)
    R = np.abs((o.intensity() - I) / dt / I).reshape(N, N, o.nd)[2:N - 2, 2:N - 2]
    return R.mean(), R.max()


def test_tolman_field_stationary_in_kerr():
    """a = 0.9, r in [6, 7], theta in [1, 1.2]: the residual of the exact
    stationary field is truncation, falling about 3x in its mean per doubling
    of the angular resolution (n = 2 -> 4 -> 8: measured 1.8e-2, 5.7e-3,
    1.7e-3).  A wrong drift sign or flux weight leaves a residual of order 0.2
    (the angular terms themselves)."""
    m2, _ = tolman_residual(2)
    m4, x4 = tolman_residual(4)
    m8, _ = tolman_residual(8)
    assert m4 < 8e-3 and x4 < 2e-2
    assert m2 / m4 > 2.8 and m4 / m8 > 2.8


def test_uniform_field_stationary_flat_spherical():
    """M = 0: flat space under the rotating spherical tetrad (section 4.5).
    n_0 = -1, so the stationary field is uniform and isotropic; its residual
    shrinks with the angular resolution as in curved space."""
    kw = dict(a=0.0, M=0.0, r0=2.0, r1=3.0, t0=0.7, t1=1.0)
    m2, _ = tolman_residual(2, **kw)
    m4, x4 = tolman_residual(4, **kw)
    m8, _ = tolman_residual(8, **kw)
    assert m4 < 6e-3 and x4 < 2e-2
    assert m2 / m4 > 2.5 and m4 / m8 > 2.5


# --------------------------------------------------------------- upwind side
def upwind_bump(mutant=0, steps=50, dt=0.05):
    """One flat spherical cell (no spatial flux): donor-cell angular transport of
    a bump in direction space; returns (min I, max I, <n_r> before, after)."""
    cfg = W.base_config(4, (1, 1, 1), (math.log(3.0), 1.1, 0.0), (0.05, 0.05, 0.05), (("periodic",) * 2,) * 3,
                        coords="kerr_schild", a=0.0, M=0.0, source=False, n0_cut=0.0, order=1, ang_recon="donor")
    o = oracle.Oracle(cfg, mutant=mutant)
    gr = o.grid()
    d, w = gr["dir"], gr["w"]
    c = np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])
    I = np.exp(-((d - c) ** 2).sum(1) / 0.05)
    o.set_fluid([0.0], [0.0], [[1, 0, 0, 0]], [0.0], [0.0])
    o.set_intensity(I[None])
    o.step(dt, steps)
    J = o.intensity()[0]
    mr = lambda X: (X * w * d[:, 0]).sum() / (X * w).sum()
    return J.min(), J.max(), mr(I), mr(J)


def test_angular_flux_is_upwind():
    """eq. angular_fluxes takes the upwind value by the sign of the drift: with
    donor-cell reconstruction the update is then a positive combination of old
    values (angular CFL about 0.1 here), so no intensity turns negative.  In
    flat space every direction turns towards the outward radial one (dm_r/ds =
    (1 - m_r^2)/r), and the mean radial cosine grows."""
    mn, mx, mr0, mr1 = upwind_bump()
    assert mn >= -1e-15 and mx <= 1.0
    assert mr1 > mr0 + 0.2


# --------------------------------------------------------------- straight beam
def tangential_beam(mutant=0, N=16, n_geo=4, r0=1.5, ph0=0.3, T=0.8):
    """Flat spherical coordinates, equatorial wedge (ln r, phi) with one theta
    cell: a packet launched along phi-hat at (r0, ph0); returns the distance of
    its energy centroid at time T from the straight line's point r0 r-hat + T phi-hat."""
    rlo, rhi, plo, phi_ = 1.0, 3.0, 0.0, 1.2
    dx = ((math.log(rhi) - math.log(rlo)) / N, 0.02, (phi_ - plo) / N)
    cfg = W.base_config(n_geo, (N, 1, N), (math.log(rlo), math.pi / 2 - 0.01, plo), dx,
                        (("outflow", "outflow"), ("periodic", "periodic"), ("outflow", "outflow")),
                        coords="kerr_schild", a=0.0, M=0.0, source=False, n0_cut=0.0)
    o = oracle.Oracle(cfg, mutant=mutant)
    g = o.grid()
    s_star = int(np.argmax(g["dir"] @ np.array([0.0, 0.0, 1.0])))   # phi-hat, an exact grid direction
    rc = np.exp(math.log(rlo) + (np.arange(N) + 0.5) * dx[0])
    pc = plo + (np.arange(N) + 0.5) * dx[2]
    X = rc[None, :] * np.cos(pc)[:, None]
    Y = rc[None, :] * np.sin(pc)[:, None]
    I = np.zeros((N * N, o.nd))
    I[:, s_star] = np.exp(-((X - r0 * math.cos(ph0)) ** 2 + (Y - r0 * math.sin(ph0)) ** 2) / (2 * 0.05 ** 2)).ravel()
    o.set_fluid(np.zeros(N * N), np.zeros(N * N), W.static_ucon(N * N), np.zeros(N * N), np.zeros(N * N))
    o.set_intensity(I)
    n = int(math.ceil(T / o.cfl_dt(0.4)))
    o.step(T / n, n)
    E = (o.intensity() @ g["w"]).reshape(N, N) * (rc ** 3)[None, :]    # sqrt(-g) = r^3 sin(theta) in ln r
    xc, yc = (E * X).sum() / E.sum(), (E * Y).sum() / E.sum()
    xe, ye = r0 * math.cos(ph0) - T * math.sin(ph0), r0 * math.sin(ph0) + T * math.cos(ph0)
    return math.hypot(xc - xe, yc - ye)


def test_tangential_beam_is_straight():
    """Section 4.5: the packet's centroid stays within two cells (0.15, cells of
    about 0.07 at r ~ 1.7) of the straight line after travelling 0.8; a drift of
    the wrong sign bends it by twice that."""
    assert tangential_beam() < 0.15


# --------------------------------------------------------------- pole boundary
def smooth_cartesian_field(x, N):
    """A field smooth in Cartesian position x and Cartesian direction N."""
    return (1.0 + 0.3 * x[..., 0] + 0.2 * x[..., 1] - 0.1 * x[..., 2]) * \
           (1.0 + 0.5 * N[..., 0] - 0.3 * N[..., 1] + 0.2 * N[..., 2])


def spherical_frame(r, th, ph):
    """Position and the legs (r-hat, theta-hat, phi-hat) of the spherical chart,
    continued analytically to theta outside [0, pi] (phi-hat = d_phi / (r sin theta))."""
    st, ct, sp, cp = math.sin(th), math.cos(th), math.sin(ph), math.cos(ph)
    rh = np.array([st * cp, st * sp, ct])
    return r * rh, rh, np.array([ct * cp, ct * sp, -st]), np.array([-sp, cp, 0.0])


def pole_ghost_error(mutant=0, nr=3, nth=6, nph=8):
    """Largest difference between the oracle's pole ghosts of a smooth field and
    the field evaluated in the continued chart (ghost rows on both poles)."""
    dx = (0.2, math.pi / nth, 2 * math.pi / nph)
    cfg = W.base_config(2, (nr, nth, nph), (math.log(1.0), 0.0, 0.0), dx,
                        (("outflow", "outflow"), ("pole", "pole"), ("periodic", "periodic")),
                        coords="kerr_schild", a=0.0, M=0.0)
    o = oracle.Oracle(cfg, mutant=mutant)
    d = o.grid()["dir"]
    def field_at(i, j, k):
        r = math.exp((i + 0.5) * dx[0]); th = (j + 0.5) * dx[1]; ph = (k + 0.5) * dx[2]
        x, rh, thh, phh = spherical_frame(r, th, ph)
        N = d[:, 0:1] * rh + d[:, 1:2] * thh + d[:, 2:3] * phh
        return smooth_cartesian_field(x[None, :], N)
    I = np.zeros((nph, nth, nr, o.nd))
    for k in range(nph):
        for j in range(nth):
            for i in range(nr):
                I[k, j, i] = field_at(i, j, k)
    G = o.ghosts(I.reshape(-1, o.nd))          # (gn2, gn1, gn0, nd), two ghost layers per active axis
    err = 0.0
    for k in range(nph):
        for j in (-2, -1, nth, nth + 1):
            for i in range(nr):
                err = max(err, np.abs(G[k + 2, j + 2, i + 2] - field_at(i, j, k)).max())
    return err


def test_pole_ghost_continues_the_chart():
    """The ghost rows beyond theta = 0 and theta = pi hold the field of the cell
    across the pole (phi + pi) seen with theta-hat and phi-hat reversed: exactly
    the smooth field of the continued chart, so the reconstruction's slopes see
    no seam at the pole (c22/c23 readings of section 5's pole treatment)."""
    assert pole_ghost_error() < 1e-13


# --------------------------------------------------------------- planted mistakes
def failed_pins(mutant):
    """Names of the pins above that an oracle build with planted mistake
    `mutant` fails."""
    checks = {
        "drift": lambda: drift_error(0.9, 1.0, 3.0, 1.1, mutant) < 1e-8,
        "stationary": lambda: tolman_residual(4, mutant=mutant)[0] < 8e-3,
        "upwind": lambda: upwind_bump(mutant)[0] >= -1e-15,
        "beam": lambda: tangential_beam(mutant) < 0.15,
        "pole": lambda: pole_ghost_error(mutant) < 1e-13,
        "orbit": lambda: orbit_turn(0.95, mutant) < -2e-4 and orbit_turn(1.05, mutant) > 2e-4,
    }
    return sorted(name for name, ok in checks.items() if not ok())


@pytest.mark.parametrize("mutant,expect", [(1, "drift"), (1, "orbit"), (2, "upwind"), (3, "pole"), (4, "pole"), (6, "drift")])
def test_planted_mistakes_are_caught(mutant, expect):
    """Mistakes planted in copies of the oracle (drift sign flipped; upwind side
    taken from the weighted speed n_0 v.u, i.e. downwind where n_0 < 0; pole
    ghost without the phi + pi shift or without the direction mirror; angular
    flux without its n_0 weight) each fail at least the named pin."""
    assert expect in failed_pins(mutant)
