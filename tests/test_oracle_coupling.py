"""Pins of the oracle's temperature solves, methods 1 and 2 of section 3.5.2
(the third, the default, is pinned in test_oracle_pins.py), on one cell of a
static fluid in flat space, where n^0 = D = 1:

* the temperature after one interaction satisfies the paper's printed
  equation: eq. semi_implicit_T (method 1, A2 alpha^a_P(T_-) a T_+^4 + ...)
  and eq. implicit_T (method 2, A2 N a sqrt(T_+) + ... for alpha^a = N T^-7/2),
  with A1 and A2 of eqs. A1, A2 restated here;
* the intensity update is eq. fluid_interaction_discrete with the explicit
  alpha_- and the emission at T_+ (Planck absorption at T_- or T_+);
* thermal equilibrium is stationary for every method;
* with a temperature-independent opacity (T^-p, p = 0) the three methods are
  the same equation and give the same step.
CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_15532_b300 import workloads as W

FOURPI = 4.0 * math.pi


def one_cell(method, T_gas=2.0, T_rad=1.0, rho=1.0, kappa=0.3, alpha_s=0.2, p=3.5, eta=1.0, n_geo=2, seed=5):
    cfg = W.base_config(n_geo, (1, 1, 1), (0, 0, 0), (1, 1, 1), (("periodic",) * 2,) * 3,
                        transport=False, coupling=method, T_exp=p, rho_exp=1.0)
    o = oracle.Oracle(cfg)
    g = o.grid()
    rng = np.random.default_rng(seed)
    I0 = W.planck(T_rad) * (1.0 + 0.2 * rng.uniform(-1, 1, o.nd))
    Y = rho / (W.GAMMA - 1.0)
    o.set_fluid([rho], [Y * T_gas], W.static_ucon(1), [kappa], [alpha_s], [eta])
    o.set_intensity(I0[None])
    return o, g, I0, Y


def step_and_state(method, dt=0.3, **kw):
    o, g, I0, Y = one_cell(method, **kw)
    fails = o.source_only(dt)
    return o, g, I0, Y, fails


@pytest.mark.parametrize("method", [1, 2])
def test_root_satisfies_the_printed_equation(method):
    T_gas, rho, kappa, alpha_s, p, dt = 2.0, 1.0, 0.3, 0.2, 3.5, 0.3
    o, g, I0, Y, fails = step_and_state(method, dt=dt, T_gas=T_gas, rho=rho, kappa=kappa, alpha_s=alpha_s, p=p)
    assert fails == 0
    w = g["w"]
    N = kappa * rho                          # alpha^a = N T^-p (rho_exp = 1)
    a_m = N * T_gas ** -p + alpha_s * rho    # explicit total absorption
    A1 = (I0 * w).sum() / (1.0 + a_m * dt)
    A2 = dt / FOURPI * w.sum() / (1.0 + a_m * dt)
    Em, a_s = (I0 * w).sum(), alpha_s * rho
    Tp = o.ug()[0] / Y
    lin = Y * (1.0 - A2 * a_s)
    if method == 1:
        terms = [A2 * N * T_gas ** -p * Tp ** 4, lin * Tp, A1, -lin * T_gas, -(1.0 - A2 * a_s) * Em]
    else:
        terms = [A2 * N * math.sqrt(Tp), lin * Tp, A1, -lin * T_gas, -(1.0 - A2 * a_s) * Em]
    assert abs(sum(terms)) < 1e-12 * max(abs(t) for t in terms)
    # the intensity update with the explicit alpha_- and the emission at T_+
    aP = N * (T_gas if method == 1 else Tp) ** -p
    Ep = Em + Y * (T_gas - Tp)
    em = aP * Tp ** 4 + a_s * Ep
    Iexp = (I0 + dt / FOURPI * em) / (1.0 + a_m * dt)
    assert np.abs(o.intensity()[0] - Iexp).max() < 1e-13 * np.abs(Iexp).max()
    # the gas took what the radiation gave
    assert abs((o.intensity()[0] * w).sum() + o.ug()[0] - (Em + Y * T_gas)) < 1e-13 * (Em + Y * T_gas)


@pytest.mark.parametrize("method", [1, 2, 3])
def test_equilibrium_is_stationary(method):
    o, g, I0, Y = one_cell(method, T_gas=1.3, T_rad=1.3)
    Ieq = np.full(o.nd, W.planck(1.3))
    o.set_intensity(Ieq[None])
    o.source_only(0.4)
    assert np.abs(o.intensity()[0] - Ieq).max() < 1e-14 * Ieq.max()
    assert abs(o.ug()[0] / Y - 1.3) < 1e-14


def test_methods_agree_for_temperature_independent_opacity():
    res = []
    for method in (1, 2, 3):
        o, g, I0, Y, fails = step_and_state(method, p=0.0, kappa=2.0, alpha_s=0.5, T_gas=1.5, dt=0.2)
        assert fails == 0
        res.append((o.intensity()[0], o.ug()[0]))
    for I, u in res[1:]:
        assert np.abs(I - res[0][0]).max() < 1e-13 * np.abs(res[0][0]).max()
        assert abs(u - res[0][1]) < 1e-13 * abs(res[0][1])
