"""Shared helpers of the parity tests: run one workload on the CUDA library
and on the FP64 oracle from the same seeded inputs."""
import math

import numpy as np

import oracle
from paper_2508_15532_b300 import workloads as W


def rel_err(x, ref, floor_frac=1e-6):
    """|x - ref| / max(|ref|, floor_frac * max|ref|), elementwise."""
    ref = np.asarray(ref, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    floor = floor_frac * max(np.abs(ref).max(), 1e-300)
    return np.abs(x - ref) / np.maximum(np.abs(ref), floor)


def run_oracle(cfg, f, dt, nsteps):
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    o.set_intensity(f["I"])
    fails = o.step(dt, nsteps)
    R, E, G = o.moments()
    return dict(I=o.intensity(), ug=o.ug(), R=R, E=E, G=G, fails=fails)


def run_gpu(cfg, f, dt, nsteps, precision="fp64", grid=None):
    import torch
    import paper_2508_15532_b300 as rt
    g = grid or rt.Grid(cfg["n_geo"])
    st = rt.RadiationStep(g, cfg, precision=precision)
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    st.set_fluid(T(f["rho"]), T(f["ug"]), T(f["ucon"]), T(f["kappa"]), T(f["alpha_s"]), T(f["eta"]))
    tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[precision]
    I0 = torch.as_tensor(np.asarray(f["I"], dtype=np.float64), device=dev).to(tdt).contiguous()
    st.set_intensity(I0)
    _, nfail = st.step(dt, nsteps, check=True)
    nc, nd = I0.shape
    I = torch.empty_like(I0)
    st.get_intensity(I)
    ug = torch.empty(nc, dtype=torch.float64, device=dev)
    st.get_ugas(ug)
    R = torch.empty(nc, 10, dtype=torch.float64, device=dev)
    E = torch.empty(nc, dtype=torch.float64, device=dev)
    G = torch.empty(nc, 4, dtype=torch.float64, device=dev)
    st.moments(R, E, G)
    torch.cuda.synchronize()
    out = dict(I=I.double().cpu().numpy(), ug=ug.cpu().numpy(), R=R.cpu().numpy(), E=E.cpu().numpy(),
               G=G.cpu().numpy(), fails=nfail)
    del st
    return out


def diffusion_closed_form(x, t, K, sigma2=W.DIFF_SIGMA2):
    """eq. diff_analytic: a Gaussian of variance sigma2 spreading under
    dE/dt = K d2E/dx2 (the paper writes K = 1 / (3 alpha^s), D = 2 K / sigma2)."""
    v = 1.0 + 2.0 * K * t / sigma2
    return v ** -0.5 * np.exp(-x * x / (2.0 * v * sigma2))


def scheme_diffusion_coefficient(dirs, w, abar=1.0, alpha=W.DIFF_ALPHA_S):
    """Thick limit of the damped face flux (eqs. rad_speeds, flux_Jiang): with
    f(tau), g(tau) -> 1/tau, direction s carries -|n^x_s| / (2 tau) (I_{l+1} - I_l)
    (pinned by test_flux_thick_limit_is_diffusive), tau = abar alpha dx.  An
    isotropic field I = E / (4 pi) then carries the energy flux
    -(sum_s |n^x_s| dOmega_s) / (8 pi abar alpha) dE/dx, i.e. K = 1 / (4 abar alpha)
    for the exact sum 2 pi: 3/4 of the continuum 1 / (3 alpha)."""
    return float(np.abs(np.asarray(dirs)[:, 0]) @ np.asarray(w)) / (8.0 * math.pi * abar * alpha)
