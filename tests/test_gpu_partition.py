"""x3 slab decomposition on the CUDA path: a box split into 2 or 3 slab
contexts on one GPU, whose ghost planes are filled before every stage from
the neighbours' halo blocks (rt_halo_pack / rt_halo_unpack, copied in this
process by partition.LocalExchange), reproduces the single-context run bit
for bit: the packed FP32/BF16 kernel, the FP64 flat kernel, the general
kernel with a moving fluid (ghost velocities from rt_set_fluid_halo) and the
Kerr-Schild band with angular fluxes.  The same exchange loop runs over
torch.distributed on several GPUs (partition.DistExchange); its index logic is
tested on CPU (tests/test_partition.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import partition as PT
from paper_2508_15532_b300 import workloads as W

pytestmark = pytest.mark.gpu

DT = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _ctx(grid, cfg, f, precision, sl=slice(None)):
    st = rt.RadiationStep(grid, cfg, precision=precision)
    st.set_fluid(*(_T(np.asarray(f[k])[sl]) for k in ("rho", "ug", "ucon", "kappa", "alpha_s", "eta")))
    st.set_intensity(torch.as_tensor(np.asarray(f["I"])[sl], device="cuda").to(DT[precision]).contiguous())
    return st


def _state(st, nc, nd, precision):
    I = torch.empty(nc, nd, dtype=DT[precision], device="cuda")
    u = torch.empty(nc, dtype=torch.float64, device="cuda")
    st.get_intensity(I)
    st.get_ugas(u)
    return I, u


def flat_case(nx=(12, 6, 12), index=81):
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + index))
    nc = int(np.prod(nx))
    rho = np.exp(rng.normal(0.0, 0.5, nc))
    T = rng.uniform(0.5, 2.0, nc)
    cfg = W.base_config(4, nx, (0, 0, 0), tuple(1.0 / n for n in nx), (("periodic", "periodic"),) * 3)
    f = dict(rho=rho, ug=rho * T / (W.GAMMA - 1.0), ucon=W.static_ucon(nc), kappa=np.full(nc, 1e-2),
             alpha_s=np.full(nc, 0.4), eta=np.ones(nc), I=W.planck(T)[:, None] * (1.0 + 0.1 * rng.uniform(-1, 1, (nc, 162))))
    return cfg, f


def moving_case():
    cfg, f = flat_case(index=82)
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + 83))
    nc = f["rho"].shape[0]
    v = rng.uniform(-0.1, 0.1, (nc, 3))
    g = 1.0 / np.sqrt(1.0 - (v * v).sum(1))
    f["ucon"] = np.concatenate([g[:, None], g[:, None] * v], axis=1)
    cfg = dict(cfg, bc=(cfg["bc"][0], cfg["bc"][1], ("outflow", "outflow")))
    return cfg, f


def kerr_band():
    cfg, f = W.kerr(nr=16, nth=8, nph=12, n_geo=4, index=84)
    cfg = dict(cfg, bc=(cfg["bc"][0], ("outflow", "outflow"), cfg["bc"][2]), n_pole_zero=0)
    return cfg, f


def split_equals_single(cfg, f, precision, world, nsteps=3):
    grid = rt.Grid(cfg["n_geo"])
    nc, nd = np.asarray(f["I"]).shape
    one = _ctx(grid, cfg, f, precision)
    dt = one.cfl_dt(0.4)
    one.step(dt, nsteps)
    I1, u1 = _state(one, nc, nd, precision)
    slabs = []
    for r in range(world):
        sl = PT.slab_cells(cfg, r, world)
        st = _ctx(grid, PT.slab_config(cfg, r, world), f, precision, sl)
        lo, hi = PT.halo_fluid(cfg, f, r, world)
        st.set_fluid_halo(lo, hi)
        slabs.append((st, sl))
    fails = PT.LocalExchange(cfg, [s for s, _ in slabs], cfg.get("order", 2)).step_all(dt, nsteps)
    assert fails == 0
    I = torch.cat([_state(s, sl.stop - sl.start, nd, precision)[0] for s, sl in slabs])
    u = torch.cat([_state(s, sl.stop - sl.start, nd, precision)[1] for s, sl in slabs])
    return torch.equal(I, I1) and torch.equal(u, u1), float((I.double() - I1.double()).abs().max())


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp64"])
@pytest.mark.parametrize("world", [2, 3])
def test_flat_box_split_is_bit_identical(precision, world):
    ok, d = split_equals_single(*flat_case(), precision, world)
    assert ok, d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_moving_fluid_split_is_bit_identical(precision):
    ok, d = split_equals_single(*moving_case(), precision, 2)
    assert ok, d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kerr_band_split_is_bit_identical(precision):
    ok, d = split_equals_single(*kerr_band(), precision, 2, nsteps=2)
    assert ok, d


def test_order_one_split_is_bit_identical():
    cfg, f = flat_case(index=85)
    ok, d = split_equals_single(dict(cfg, order=1), f, "fp32", 2)
    assert ok, d


def test_halo_context_refuses_whole_steps():
    cfg, f = flat_case(index=86)
    st = _ctx(rt.Grid(4), PT.slab_config(cfg, 0, 2), f, "fp32", PT.slab_cells(cfg, 0, 2))
    with pytest.raises(rt.RTError) as e:
        st.step(1e-3, 1)
    assert e.value.status == 1
    with pytest.raises(rt.RTError) as e:
        st.step_stage(1e-3, 1)
    assert e.value.status == 5
