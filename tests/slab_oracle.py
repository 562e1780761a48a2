"""The oracle as a slab stepper of paper_2508_15532_b300.partition (halo pack,
ghost-plane buffers, unpack, stage), for the CPU tests of the x3 domain
decomposition."""
import numpy as np
import torch

import oracle
from paper_2508_15532_b300 import partition as PT


class OracleSlab:
    def __init__(self, cfg, fields, rank, world):
        self.cfg = PT.slab_config(cfg, rank, world)
        sl = PT.slab_cells(cfg, rank, world)
        self.o = oracle.Oracle(self.cfg)
        f = {k: np.asarray(v)[sl] for k, v in fields.items() if k in ("rho", "ug", "ucon", "kappa", "alpha_s", "eta", "I")}
        self.o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
        self.o.set_intensity(f["I"])
        if world > 1:
            lo, hi = PT.halo_fluid(cfg, fields, rank, world)
            self.o.set_fluid_halo(lo, hi)
            n = self.o.halo_doubles()
            self.rbuf = (torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64))

    def halo_pack(self, stage):
        lo, hi = self.o.halo_pack(stage)
        return torch.from_numpy(lo), torch.from_numpy(hi)

    def halo_recv_buffers(self):
        return self.rbuf

    def halo_unpack(self, lo, hi):
        self.o.halo_unpack(lo.numpy(), hi.numpy())

    def step_stage(self, dt, stage):
        return self.o.step_stage(dt, stage)
