"""x3 slab decomposition of the step (the spatial domain decomposition along
x3): the oracle split into slabs, with the two ghost planes per side
exchanged before every stage, reproduces the single-domain oracle bit for
bit.  In one process (LocalExchange, world 2 and 3) and across gloo ranks
(DistExchange over torch.distributed point-to-point, world 2 and 3), on a
periodic box with the opacity/coupling fields, on an outflow box with a
moving fluid (the ghost fluid enters the face opacity and the advective
term), and on a Kerr-Schild band with angular fluxes.  CPU only."""
import math
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2508_15532_b300 import partition as PT
from paper_2508_15532_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_slab_ranges_cover_the_box():
    for nz, world in ((12, 2), (12, 3), (13, 4), (8, 4)):
        r = [PT.slab_range(nz, k, world) for k in range(world)]
        assert r[0][0] == 0 and r[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert all(k1 - k0 >= 2 for k0, k1 in r)
    with pytest.raises(ValueError):
        PT.slab_range(5, 0, 3)


def test_slab_configs():
    cfg = W.base_config(2, (4, 4, 12), (0, 0, 0), (0.25, 0.25, 1 / 12), (("periodic", "periodic"),) * 3)
    c1 = PT.slab_config(cfg, 1, 3)
    assert c1["nx"] == (4, 4, 4) and c1["bc"][2] == ("halo", "halo") and abs(c1["x0"][2] - 4 / 12) < 1e-15
    assert PT.neighbours(cfg, 0, 3) == (2, 1) and PT.neighbours(cfg, 2, 3) == (1, 0)
    co = dict(cfg, bc=(cfg["bc"][0], cfg["bc"][1], ("outflow", "outflow")))
    assert PT.neighbours(co, 0, 3) == (None, 1) and PT.neighbours(co, 2, 3) == (1, None)
    assert PT.slab_config(co, 0, 3)["bc"][2] == ("outflow", "halo")
    assert PT.slab_config(co, 2, 3)["bc"][2] == ("halo", "outflow")


def case_periodic():
    cfg, f = W.flat3d(N=6, n_geo=2, index=71)
    cfg = dict(cfg, nx=(6, 6, 6))
    return cfg, f, 3


def case_moving_outflow():
    """outflow x3 faces, a seeded velocity field (|v| <= 0.1)"""
    rng = np.random.Generator(np.random.PCG64(W.SEED0 + 72))
    nx = (5, 4, 9)
    nc = int(np.prod(nx))
    cfg = W.base_config(2, nx, (0, 0, 0), (0.2, 0.25, 1 / 9),
                        (("periodic", "periodic"), ("periodic", "periodic"), ("outflow", "outflow")))
    rho = np.exp(rng.normal(0.0, 0.5, nc))
    T = rng.uniform(0.5, 2.0, nc)
    v = rng.uniform(-0.1, 0.1, (nc, 3))
    g = 1.0 / np.sqrt(1.0 - (v * v).sum(1))
    ucon = np.concatenate([g[:, None], g[:, None] * v], axis=1)
    f = dict(rho=rho, ug=rho * T / (W.GAMMA - 1.0), ucon=ucon, kappa=np.full(nc, 1e-2), alpha_s=np.full(nc, 0.4),
             eta=np.ones(nc), I=W.planck(T)[:, None] * (1.0 + 0.1 * rng.uniform(-1, 1, (nc, 42))))
    return cfg, f, 3


def case_kerr_band():
    """Kerr-Schild a = 0.9 torus fields on a theta band (outflow theta faces,
    no pole), phi periodic and split: angular fluxes and the boosted
    interaction across slab faces"""
    cfg, f = W.kerr(nr=10, nth=6, nph=8, n_geo=2, index=73)
    cfg = dict(cfg, bc=(cfg["bc"][0], ("outflow", "outflow"), cfg["bc"][2]), n_pole_zero=0)
    return cfg, f, 2


CASES = {"periodic": case_periodic, "moving_outflow": case_moving_outflow, "kerr_band": case_kerr_band}


def single_domain(cfg, f, nsteps):
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    o.set_intensity(f["I"])
    dt = o.cfl_dt(0.4)
    assert o.step(dt, nsteps) == 0
    return dt, o.intensity(), o.ug()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("world", [2, 3])
def test_oracle_split_in_process_is_bit_identical(name, world):
    from slab_oracle import OracleSlab
    cfg, f, nsteps = CASES[name]()
    if cfg["nx"][2] < 2 * world:
        pytest.skip("box too thin for this split")
    dt, I_ref, u_ref = single_domain(cfg, f, nsteps)
    slabs = [OracleSlab(cfg, f, r, world) for r in range(world)]
    assert PT.LocalExchange(cfg, slabs, cfg.get("order", 2)).step_all(dt, nsteps) == 0
    I = np.concatenate([s.o.intensity() for s in slabs])
    u = np.concatenate([s.o.ug() for s in slabs])
    assert np.array_equal(I, I_ref) and np.array_equal(u, u_ref)


def test_halo_is_needed():
    """Without the exchange (ghost planes left at zero) the split differs:
    the comparison above sees the halo."""
    from slab_oracle import OracleSlab
    cfg, f, nsteps = case_periodic()
    dt, I_ref, _ = single_domain(cfg, f, nsteps)
    slabs = [OracleSlab(cfg, f, r, 2) for r in range(2)]
    for _ in range(nsteps):
        for stage in (0, 1):
            for s in slabs:
                s.step_stage(dt, stage)
    I = np.concatenate([s.o.intensity() for s in slabs])
    assert not np.array_equal(I, I_ref)


def _gloo_worker(rank, world, port, name, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from slab_oracle import OracleSlab
        cfg, f, nsteps = CASES[name]()
        o = oracle.Oracle(cfg)
        dt = o.cfl_dt(0.4)
        del o
        s = OracleSlab(cfg, f, rank, world)
        fails = PT.SlabDriver(s, PT.DistExchange(cfg, rank, world), cfg.get("order", 2)).step(dt, nsteps)
        q.put((rank, fails, s.o.intensity(), s.o.ug()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("periodic", 2), ("moving_outflow", 3), ("kerr_band", 2)])
def test_oracle_split_over_gloo_ranks_is_bit_identical(name, world):
    cfg, f, nsteps = CASES[name]()
    dt, I_ref, u_ref = single_domain(cfg, f, nsteps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() * 7 + world) % 400
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, fails, I, u = q.get(timeout=300)
        res[r] = (fails, I, u)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(res[r][0] == 0 for r in res)
    I = np.concatenate([res[r][1] for r in range(world)])
    u = np.concatenate([res[r][2] for r in range(world)])
    assert np.array_equal(I, I_ref) and np.array_equal(u, u_ref)
