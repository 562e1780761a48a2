"""The adjoint workload as stated: 64^3 cells, 162 directions, a 64-step
rollout with a checkpoint every 8 steps, loss L = sum_c E_c^2 of the final
comoving energy density.  Gradients in the absorption prefactor kappa, the
emission multiplier eta and the initial intensity I_0 from the checkpointed
rollout (FP64 and mixed FP32/FP64) against central finite differences of the
CUDA FP64 forward at 32 seeded cells (I_0: 32 seeded (cell, direction)
pairs).

Step sizes.  At h = 1e-6 (relative) the quotient's own rounding noise is
about 1e-4 of it: the perturbation moves every energy density of the box
(64 steps reach 256 cells, the whole periodic box), and each of the 262,144
differences E+ - E- carries FP64 rounding of ~1e-14 E against a change of
~1e-8 E.  The FP64 and the mixed gradients then differ from the quotient by
the same amounts (measured: medians 2e-5, largest 1.4e-4 to 2.9e-4 for both),
which is the quotient's noise, not the gradients' error.  The quotient at
h = 1e-4 has 100 times less noise and a truncation error of ~h^2 = 1e-8, so
the 1e-5 bar is held there, on all 32 samples; h = 1e-6 is run on the first
8 samples and held to 1e-3.

The quotient's noise is absolute, not relative to the component: over the
32 eta samples the spread between the quotients at h = 1e-4, 3e-5 and 1e-5
puts it at 1.1e-8 (median) to 4.5e-8 (largest) at h = 1e-4, about 2e-7 of
the largest gradient, and the gradients' absolute errors measure the same
(median 1.7e-8, largest 3.8e-8).  Against a component of 1% of the largest
that noise alone is 2e-5 relative.  So components are compared relative to
max(|quotient|, 3e-2 of the largest component), where the largest noise
stays below 1e-5 at h = 1e-4 and below 1e-3 at h = 1e-6.

Bars: FP64 gradients within 1e-5 of the quotient (h = 1e-4); the mixed
gradients (FP32 per-element reverse arithmetic, FP64 per-cell sums) within
1e-3.  RT_REPORT_DIR, when set, receives the measured errors as JSON."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import workloads as W
from paper_2508_15532_b300.rollout import rollout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_adjoint_workload_32_cells_central_differences():
    cfg, f = W.adjoint3d(N=64, n_geo=4)
    nsteps, ck = cfg["nsteps"], cfg["ckpt_every"]
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    g = rt.Grid(cfg["n_geo"])
    wt = T(g.query()[1])
    fluid = dict(rho=T(f["rho"]), ucon=T(f["ucon"]), alpha_s=T(f["alpha_s"]))
    ug0 = T(f["ug"])
    grads = {}
    dt = None
    for prec in ("fp64", "fp32"):
        st = rt.RadiationStep(g, cfg, precision=prec)
        dt = st.cfl_dt(0.4) if dt is None else dt
        I0 = T(f["I"]) if prec == "fp64" else T(f["I"]).float()
        I0.requires_grad_()
        kappa = T(f["kappa"]).requires_grad_()
        eta = T(f["eta"]).requires_grad_()
        IN, _ = rollout(st, fluid, I0, ug0, kappa, eta, nsteps, dt=dt, ckpt_every=ck)
        ((IN.double() @ wt) ** 2).sum().backward()
        grads[prec] = {"kappa": kappa.grad.detach().clone(), "eta": eta.grad.detach().clone(),
                       "I0": I0.grad.detach().double().clone()}
        del st, IN
    torch.cuda.empty_cache()

    fw = rt.RadiationStep(g, cfg, precision="fp64")
    base = {"kappa": T(f["kappa"]), "eta": T(f["eta"]), "I0": T(f["I"])}

    def energy(which, c, s, h):
        p = {k: v for k, v in base.items()}
        p[which] = base[which].clone()
        if which == "I0":
            p["I0"][c, s] += h
        else:
            p[which][c] += h
        fw.set_fluid(fluid["rho"], ug0, fluid["ucon"], p["kappa"], fluid["alpha_s"], p["eta"])
        fw.set_intensity(p["I0"])
        _, nf = fw.step(dt, nsteps, check=True)
        assert nf == 0
        I = torch.empty_like(p["I0"])
        fw.get_intensity(I)
        return I @ wt

    rng = np.random.default_rng(20250815)
    nc, nd = f["I"].shape
    cells = rng.choice(nc, 32, replace=False)
    dirs = rng.integers(0, nd, 32)
    out = {}
    for rel_h, nsamp in ((1e-4, 32), (1e-6, 8)):
        for which in ("kappa", "eta", "I0"):
            rows = []
            for c, s in list(zip(cells, dirs))[:nsamp]:
                b = float(base[which][c, s]) if which == "I0" else float(base[which][c])
                h = rel_h * b
                Ep, Em = energy(which, c, s, h), energy(which, c, s, -h)
                # L(+) - L(-) = sum (E+ - E-)(E+ + E-): no cancellation in the sum
                fd = float(((Ep - Em) * (Ep + Em)).sum()) / (2 * h)
                idx = (int(c), int(s)) if which == "I0" else int(c)
                rows.append((fd, float(grads["fp64"][which][idx]), float(grads["fp32"][which][idx])))
            rows = np.array(rows)
            scale = max(float(grads["fp64"][which].abs().max()), 1e-300)
            den = np.maximum(np.abs(rows[:, 0]), 3e-2 * scale)
            e64 = np.abs(rows[:, 1] - rows[:, 0]) / den
            e32 = np.abs(rows[:, 2] - rows[:, 0]) / den
            e6432 = np.abs(rows[:, 2] - rows[:, 1]) / den
            out["%s_h%g" % (which, rel_h)] = dict(
                samples=int(nsamp), fp64_max=float(e64.max()), fp64_median=float(np.median(e64)),
                mixed_max=float(e32.max()), mixed_median=float(np.median(e32)),
                mixed_vs_fp64_max=float(e6432.max()), largest_gradient=scale,
                fd_min_abs=float(np.abs(rows[:, 0]).min()))
    d = os.environ.get("RT_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "adjoint_fd_32_cells.json"), "w") as fh:
            json.dump(out, fh, indent=1)
    for key, r in out.items():
        if key.endswith("h0.0001"):
            assert r["fp64_max"] <= 1e-5, (key, r)
            assert r["mixed_max"] <= 1e-3, (key, r)
        else:
            assert r["fp64_max"] <= 1e-3 and r["mixed_max"] <= 1e-3, (key, r)
