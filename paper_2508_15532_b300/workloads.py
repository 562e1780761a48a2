"""Seeded synthetic workloads shaped like the paper's test problems and its
accretion-torus run.

This module builds configuration dictionaries and input fields only; it holds
none of the radiation step's arithmetic, and both the CUDA library and the CPU
oracle read what it returns.  Seeds are ``20250815 + workload index`` through
numpy's PCG64.

Workloads (sizes are the defaults; smaller variants keep the same recipe):

* ``beam2d``   flat 2D Cartesian 32x32 cells on [0,1]^2, 42 directions, vacuum,
               one beam injected through the x1-lower face (rows 12..19) along
               the direction closest to (cos 30, sin 30, 0); 100 steps, CFL 0.4.
* ``flat3d``   flat 3D periodic 128^3 on [0,1)^3, 162 directions, static fluid,
               lognormal density (sigma 1), T ~ U[0.5, 2] per cell,
               alpha^a = 1e-2 rho T^-3.5, alpha^s = 0.4 rho,
               I = B(T) (1 + 0.1 U(-1,1)) per cell and direction.
* ``kerr2d``   Kerr-Schild a = 0.9, 256 (ln r on [0.95 r_h, 50]) x 128 (theta)
               x 1 (phi) cells, 162 directions, constant-angular-momentum
               hydrostatic torus (inner edge 6, pressure maximum 12) with
               Keplerian-like rotation and 1% density noise, Kramers-like
               free-free absorption plus electron scattering, I = B(T).
* ``kerr3d``   the same in 3D with 128 phi cells and 5% density/temperature noise.
* ``adjoint3d`` the flat3d recipe at 64^3 (rollout of 64 steps, checkpoint every 8).
* ``diffusion1d`` the static-diffusion slab of section 4: flat 1D, 64 cells on
               [-1, 1] with outflow ends, 162 directions, rho = 1, pure
               scattering alpha^s = 1e3 (no absorption, cold gas u_g = 1e-10),
               isotropic I = E0 / (4 pi) with E0 = exp(-x^2 / (2 sigma^2)),
               sigma^2 = 1.25e-2, held at E0(0.5) for |x| > 0.5; t = 10.
               With v = 0.05: the advection-diffusion variant, the slab moving
               along x and the profile centred on x = -0.5.
"""
import math

import numpy as np

SEED0 = 20250815
GAMMA = 5.0 / 3.0
ARAD = 1.0


def _rng(index):
    return np.random.Generator(np.random.PCG64(SEED0 + index))


def planck(T):
    """Frequency-integrated Planck intensity B = a T^4 / (4 pi) (scale-free units)."""
    return ARAD * np.asarray(T) ** 4 / (4.0 * math.pi)


def base_config(n_geo, nx, x0, dx, bc, **kw):
    cfg = dict(n_geo=n_geo, nx=tuple(int(v) for v in nx), x0=tuple(float(v) for v in x0),
               dx=tuple(float(v) for v in dx), bc=tuple(tuple(b) for b in bc), coords="minkowski",
               M=1.0, a=0.0, beam_dir=-1, beam_lo=0, beam_hi=0, beam_I=0.0, n_pole_zero=0,
               gam=GAMMA, arad=ARAD, rho_exp=1.0, T_exp=3.5, rho_floor=5e-4, abar=1.0, tau_dt=False,
               order=2, limiter="mc", ang_recon="mapr", transport=True, source=True, n0_cut=0.1,
               cfl=0.4)
    cfg.update(kw)
    return cfg


def static_ucon(ncell):
    u = np.zeros((ncell, 4))
    u[:, 0] = 1.0
    return u


# ------------------------------------------------------------------ beam2d
def beam2d(dirs, N=32, n_geo=2):
    """Vacuum beam test. ``dirs`` are the grid directions (canonical order)."""
    target = np.array([math.cos(math.radians(30.0)), math.sin(math.radians(30.0)), 0.0])
    s_star = int(np.argmax(np.asarray(dirs) @ target))
    lo, hi = (12 * N) // 32, (20 * N) // 32
    cfg = base_config(n_geo, (N, N, 1), (0, 0, 0), (1.0 / N, 1.0 / N, 1.0),
                      (("beam", "outflow"), ("outflow", "outflow"), ("periodic", "periodic")),
                      beam_dir=s_star, beam_lo=lo, beam_hi=hi, beam_I=1.0, nsteps=100, workload="beam2d")
    nc = N * N
    nd = len(dirs)
    fields = dict(rho=np.zeros(nc), ug=np.zeros(nc), ucon=static_ucon(nc), kappa=np.zeros(nc),
                  alpha_s=np.zeros(nc), eta=np.ones(nc), I=np.zeros((nc, nd)))
    return cfg, fields


# ------------------------------------------------------------------ flat3d
def gaussian_field(rng, shape, sigma_cells=2.0):
    """Unit-variance Gaussian random field: white noise smoothed by a Gaussian
    kernel of ``sigma_cells`` through the FFT, then renormalised."""
    w = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) for n in shape]
    K2 = sum(np.meshgrid(*[kk ** 2 for kk in k], indexing="ij"))
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-2.0 * math.pi ** 2 * sigma_cells ** 2 * K2)))
    g -= g.mean()
    return g / g.std()


def flat3d(N=128, n_geo=4, nd=None, index=1, intensity_dtype=np.float64, with_intensity=True):
    """Periodic static-fluid box of the opacity/coupling workload.
    Arrays are cell-major with x1 fastest: cell = (k*N + j)*N + i."""
    rng = _rng(index)
    cfg = base_config(n_geo, (N, N, N), (0, 0, 0), (1.0 / N,) * 3, (("periodic", "periodic"),) * 3,
                      nsteps=100, workload="flat3d")
    nd = 10 * n_geo * n_geo + 2 if nd is None else nd
    g = gaussian_field(rng, (N, N, N))              # axes (k, j, i)
    rho = np.exp(g - 0.5).ravel()
    T = rng.uniform(0.5, 2.0, N ** 3)
    ug = rho * T / (GAMMA - 1.0)
    nc = N ** 3
    fields = dict(rho=rho, ug=ug, ucon=static_ucon(nc), kappa=np.full(nc, 1e-2),
                  alpha_s=np.full(nc, 0.4), eta=np.ones(nc), T=T)
    if with_intensity:
        I = rng.uniform(-1.0, 1.0, (nc, nd)).astype(intensity_dtype)
        I *= 0.1
        I += 1.0
        I *= planck(T).astype(intensity_dtype)[:, None]
        fields["I"] = I
    return cfg, fields


def adjoint3d(N=64, n_geo=4, **kw):
    cfg, f = flat3d(N=N, n_geo=n_geo, index=4, **kw)
    cfg.update(nsteps=64, ckpt_every=8, workload="adjoint3d")
    return cfg, f


# ------------------------------------------------------------------ Kerr torus
def _bl_metric(r, th, a, M=1.0):
    """Boyer-Lindquist g_tt, g_tphi, g_phiphi (they coincide with the
    Kerr-Schild ones); used only to shape and normalise the synthetic fluid."""
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    delta = r * r - 2 * M * r + a * a
    A = (r * r + a * a) ** 2 - a * a * delta * s2
    return -(1.0 - 2 * M * r / sig), -2 * M * a * r * s2 / sig, A * s2 / sig


def _minus_ut(r, th, a, ell):
    gtt, gtp, gpp = _bl_metric(r, th, a)
    num = gtp * gtp - gtt * gpp
    den = gpp + 2 * ell * gtp + ell * ell * gtt
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.sqrt(num / den)


def torus_fields(r, th, a, rng, r_in=6.0, r_max=12.0, noise_rho=0.01, noise_T=0.0):
    """Constant specific angular momentum hydrostatic torus with its pressure
    maximum at r_max and inner edge at r_in; rho_max = 1, p = K rho^Gamma."""
    Om = 1.0 / (r_max ** 1.5 + a)
    gtt, gtp, gpp = _bl_metric(np.array(r_max), np.array(math.pi / 2), a)
    ell = float(-(gtp + Om * gpp) / (gtt + Om * gtp))
    W_in = math.log(float(_minus_ut(np.array(r_in), np.array(math.pi / 2), a, ell)))
    with np.errstate(invalid="ignore", divide="ignore"):
        W = np.log(_minus_ut(r, th, a, ell))
    W_c = math.log(float(_minus_ut(np.array(r_max), np.array(math.pi / 2), a, ell)))
    inside = np.isfinite(W) & (W < W_in) & (r >= r_in)
    h = np.where(inside, np.exp(np.where(inside, W_in - W, 0.0)), 1.0)
    hmax = math.exp(W_in - W_c)
    K = (hmax - 1.0) * (GAMMA - 1.0) / GAMMA
    rho = np.zeros_like(r)
    rho[inside] = ((h[inside] - 1.0) * (GAMMA - 1.0) / (K * GAMMA)) ** (1.0 / (GAMMA - 1.0))
    rho = rho * (1.0 + noise_rho * rng.uniform(-1.0, 1.0, r.shape))
    Tnoise = 1.0 + noise_T * rng.uniform(-1.0, 1.0, r.shape)
    ug = K * np.abs(rho) ** GAMMA / (GAMMA - 1.0) * Tnoise
    inside &= rho > 1e-3
    atm = ~inside
    rho[atm] = 1e-4 * r[atm] ** -1.5
    ug[atm] = 1e-6 * r[atm] ** -2.5
    return rho, ug, inside


def _ks_ucon(r, th, a, Om, inside):
    """Coordinate 4-velocity in logical Kerr-Schild (t, ln r, theta, phi):
    rotation u^phi = Omega u^t in the torus, the normal observer elsewhere."""
    M = 1.0
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    z = 2 * M * r / sig
    gtt, gtp, gpp = -(1 - z), -z * a * s2, s2 * (sig + a * a * s2 * (1 + z))
    u = np.zeros(r.shape + (4,))
    norm = -(gtt + 2 * Om * gtp + Om * Om * gpp)
    ut = 1.0 / np.sqrt(np.where(inside & (norm > 0), norm, 1.0))
    # normal observer of Kerr-Schild: u^mu = -g^{t mu} / sqrt(-g^{tt}) with
    # g^{tt} = -(1 + z), g^{tr} = z, g^{t phi} = 0; u^(ln r) = u^r / r
    lapse_inv = np.sqrt(1 + z)
    u[..., 0] = np.where(inside, ut, lapse_inv)
    u[..., 1] = np.where(inside, 0.0, -z / lapse_inv / r)
    u[..., 3] = np.where(inside, Om * ut, 0.0)
    return u


def kerr(nr=256, nth=128, nph=1, n_geo=4, a=0.9, index=2, noise_rho=None, noise_T=None,
         tau_abs_max=10.0, tau_es_max=1.0, nd=None):
    """Kerr-Schild torus workload; ``nph == 1`` is the axisymmetric one."""
    rng = _rng(index)
    rh = 1.0 + math.sqrt(1.0 - a * a)
    r0, r1 = 0.95 * rh, 50.0
    dx1 = (math.log(r1) - math.log(r0)) / nr
    dx2 = math.pi / nth
    dx3 = 2 * math.pi / nph
    if noise_rho is None:
        noise_rho = 0.01 if nph == 1 else 0.05
    if noise_T is None:
        noise_T = 0.0 if nph == 1 else 0.05
    cfg = base_config(n_geo, (nr, nth, nph), (math.log(r0), 0.0, 0.0), (dx1, dx2, dx3),
                      (("outflow", "outflow"), ("pole", "pole"), ("periodic", "periodic")),
                      coords="kerr_schild", M=1.0, a=a, n_pole_zero=4, rho_exp=2.0, T_exp=3.5,
                      nsteps=200 if nph == 1 else 100, workload="kerr2d" if nph == 1 else "kerr3d")
    x1 = math.log(r0) + (np.arange(nr) + 0.5) * dx1
    x2 = (np.arange(nth) + 0.5) * dx2
    _, K2, K1 = np.meshgrid(np.arange(nph), x2, x1, indexing="ij")
    r, th = np.exp(K1), K2
    rho, ug, inside = torus_fields(r, th, a, rng, noise_rho=noise_rho, noise_T=noise_T)
    Om = 1.0 / ((r * np.sin(th)) ** 1.5 + a)
    ucon = _ks_ucon(r, th, a, Om, inside)
    T = (GAMMA - 1.0) * ug / rho
    # opacity constants: largest per-cell optical depth (radial size r dx1) of
    # absorption 10 and of scattering 1 inside the torus
    dl = r * dx1
    C_ff = tau_abs_max / (rho ** 2 * T ** -3.5 * dl)[inside].max()
    C_es = tau_es_max / (rho * dl)[inside].max()
    nc = nr * nth * nph
    nd = 10 * n_geo * n_geo + 2 if nd is None else nd
    cfg.update(C_ff=float(C_ff), C_es=float(C_es))
    fields = dict(rho=rho.ravel(), ug=ug.ravel(), ucon=ucon.reshape(nc, 4), kappa=np.full(nc, C_ff),
                  alpha_s=np.full(nc, C_es), eta=np.ones(nc), T=T.ravel())
    fields["I"] = np.repeat(planck(T.ravel())[:, None], nd, axis=1)
    return cfg, fields


def kerr2d(**kw):
    return kerr(nph=1, index=2, **kw)


def kerr3d(**kw):
    kw.setdefault("nph", 128)
    return kerr(index=3, **kw)


# ------------------------------------------------------------------ diffusion1d
DIFF_SIGMA2 = 1.25e-2
DIFF_ALPHA_S = 1e3


def diffusion1d(N=64, n_geo=4, ug=1e-10, v=0.0):
    """Static radiative diffusion through a scattering slab (section 4): the
    initial energy density, held constant beyond |x - x_c| = 0.5, and an
    isotropic intensity carrying it.  Returns (cfg, fields, x) with x the cell
    centres.  Without absorption the gas temperature does not enter the
    radiation; ``ug`` other than the cold 1e-10 serves FP32 storage, whose
    energy ledger carries an absolute rounding of ~1e-7 E-bar per stage.
    ``v`` != 0: the advection-diffusion variant, the slab moving with
    u = gamma (1, v, 0, 0) and the profile centred on x_c = -0.5 (x_c = 0 at rest)."""
    dx = 2.0 / N
    cfg = base_config(n_geo, (N, 1, 1), (-1.0, 0.0, 0.0), (dx, 1.0, 1.0),
                      (("outflow", "outflow"), ("periodic", "periodic"), ("periodic", "periodic")),
                      workload="diffusion1d" if v == 0.0 else "advection_diffusion1d")
    x = -1.0 + (np.arange(N) + 0.5) * dx
    xs = x if v == 0.0 else x + 0.5
    E0 = np.exp(-np.minimum(xs * xs, 0.25) / (2.0 * DIFF_SIGMA2))
    nd = 10 * n_geo * n_geo + 2
    ucon = static_ucon(N)
    if v != 0.0:
        gam = 1.0 / math.sqrt(1.0 - v * v)
        ucon[:, 0] = gam
        ucon[:, 1] = gam * v
    fields = dict(rho=np.ones(N), ug=np.full(N, float(ug)), ucon=ucon, kappa=np.zeros(N),
                  alpha_s=np.full(N, DIFF_ALPHA_S), eta=np.ones(N),
                  I=np.outer(E0 / (4.0 * math.pi), np.ones(nd)))
    return cfg, fields, x
