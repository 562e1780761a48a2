"""The unit scale of section 3.5.1 (eq. unit_scale) as an input transform
(paper_2508_15532_b300/units.py), pinned on the CPU:

* closed forms: GM_sun/c^2 = 1.4766 km, GM_sun/c^3 = 4.9255 microseconds;
* the paper's torus (section 5): Mdot = 1.4e18 g/s is 10% of the Eddington
  rate of a 10 M_sun hole (radiative efficiency 0.1);
* the dimensional reading rho_unit = M_unit / l_unit^3;
* a physical equilibration: one cell of gas at rho = 1 g/cm^3, T_gas = 4e7 K
  and radiation at T_rad = 1e7 K (energies of the same order), posed in code
  units through the transform and stepped by the oracle, reaches the
  temperature that energy conservation fixes in cgs, a T^4 + rho k_B T /
  ((Gamma - 1) mu m_p) = const, solved here in cgs by bisection.  A transform
  with a wrong temperature or energy scale moves that temperature."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_15532_b300 import units as U
from paper_2508_15532_b300 import workloads as W

FOURPI = 4.0 * math.pi


def test_solar_length_and_time_units():
    s = U.UnitScale(1.0, 1.0)
    assert abs(s.l_unit / 1.47662504e5 - 1.0) < 1e-7
    assert abs(s.t_unit / 4.92549095e-6 - 1.0) < 1e-7


def test_torus_accretion_rate_is_ten_percent_eddington():
    s = U.UnitScale(10.0, 1.4e18)
    assert abs(0.1 * s.mdot_eddington(0.1) / 1.4e18 - 1.0) < 0.02


def test_density_unit_reading():
    s = U.UnitScale(10.0, 1.4e18)
    assert abs(s.rho_unit * s.l_unit ** 3 / (s.Mdot * s.t_unit) - 1.0) < 1e-14
    assert abs(s.u_unit / (s.rho_unit * U.C_CGS ** 2) - 1.0) < 1e-14
    with pytest.raises(ValueError):
        U.UnitScale(0.0, 1.0)


def physical_cell(gam=5.0 / 3.0, rho_cgs=1.0, Tg_K=4e7, Tr_K=1e7, alpha_cgs=3e-6, n_geo=2):
    """One cell posed in code units through the transform; returns (scale,
    cfg, fields, W_cgs) with W_cgs the cell's total energy density in cgs."""
    s = U.UnitScale(10.0, 1.4e18)
    rho = rho_cgs / s.rho_unit
    Tg, Tr = s.temperature_code(Tg_K), s.temperature_code(Tr_K)
    a = s.arad_code()
    cfg = W.base_config(n_geo, (1, 1, 1), (0, 0, 0), (1, 1, 1), (("periodic",) * 2,) * 3, gam=gam,
                        rho_exp=0.0, T_exp=0.0, **s.config_fields())
    assert cfg["arad"] == a
    nd = 10 * n_geo * n_geo + 2
    f = dict(rho=np.array([rho]), ug=np.array([rho * Tg / (gam - 1)]), ucon=W.static_ucon(1),
             kappa=np.array([s.absorption_prefactor(alpha_cgs, 0.0, 0.0)]), alpha_s=np.zeros(1), eta=np.ones(1),
             I=np.full((1, nd), a * Tr ** 4 / FOURPI))
    W_cgs = U.A_RAD * Tr_K ** 4 + rho_cgs * U.K_B * Tg_K / ((gam - 1) * s.mu * U.M_P)
    return s, cfg, f, W_cgs


def equilibrium_K(W_cgs, rho_cgs=1.0, gam=5.0 / 3.0, mu=1.0):
    g = lambda T: U.A_RAD * T ** 4 + rho_cgs * U.K_B * T / ((gam - 1) * mu * U.M_P) - W_cgs
    lo, hi = 0.0, 1e9
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if g(mid) < 0 else (lo, mid)
    return 0.5 * (lo + hi)


def test_physical_equilibration_on_the_oracle():
    s, cfg, f, W_cgs = physical_cell()
    T_eq = equilibrium_K(W_cgs)
    assert 1e7 < T_eq < 4e7
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    o.set_intensity(f["I"])
    # alpha^a = 3e-6 / cm is 4.4 per code length: dt = 2 is alpha dt ~ 9
    for _ in range(40):
        o.source_only(2.0)
    _, E, _ = o.moments()
    Tg = (cfg["gam"] - 1) * o.ug()[0] / f["rho"][0]
    assert abs(s.temperature_K(Tg) / T_eq - 1.0) < 1e-9
    assert abs(E[0] * s.u_unit / (U.A_RAD * T_eq ** 4) - 1.0) < 1e-8
