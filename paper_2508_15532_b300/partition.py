"""Spatial domain decomposition of the radiation step into x3 slabs.

The transport couples a cell to two cells on each side per axis (the
piecewise-linear reconstruction of section 3.4 behind the face fluxes of
eqs. spatial_fluxes_vacuum and flux_Jiang); the angular flux and the
interaction are cell-local.  A box split into slabs along x3 therefore needs,
before each stage of section 3.6's predictor-corrector, one exchange with
each x3 neighbour: the two owned boundary planes of the stage's source
(intensities and what the face opacity needs).  Cells are x1-fastest, so a
plane is contiguous and the exchange moves two contiguous blocks per side.

This module holds the index arithmetic and the exchange loop only:
* slab_config / slab_range: the sub-box a rank owns, with 'halo' on the x3 faces that border another slab;
* SlabDriver: steps a slab stepper through the stages, exchanging before each
  one.  A stepper provides halo_pack(stage) -> (lo, hi), halo_unpack(lo, hi)
  and step_stage(dt, stage) (RadiationStep does, on the CUDA library);
* Exchange backends: DistExchange (torch.distributed point-to-point, NCCL
  for device buffers or gloo for host buffers) and LocalExchange (every slab
  in one process, e.g. several contexts on one GPU).
The global x3 faces keep their boundary: periodic wraps the ring of ranks,
outflow stays outflow on the first and last slab.
"""


def slab_range(nz, rank, world):
    """Owned x3 planes [k0, k1) of `rank`: as even a split as possible, each
    slab at least two planes (the depth of the halo)."""
    if world < 1 or nz < 2 * world:
        raise ValueError("x3 split: need at least 2 planes per slab (nz=%d, world=%d)" % (nz, world))
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def neighbours(cfg, rank, world):
    """(lower, upper) neighbour ranks along x3; None where the slab face is the
    box's own (non-periodic) boundary."""
    per = cfg["bc"][2][0] == "periodic"
    lo = rank - 1 if rank > 0 else (world - 1 if per else None)
    hi = rank + 1 if rank < world - 1 else (0 if per else None)
    return lo, hi


def slab_config(cfg, rank, world):
    """The rank's sub-box: its x3 planes, its x3 origin, and 'halo' on each x3
    face that borders another slab."""
    if world == 1:
        return dict(cfg)
    nz = cfg["nx"][2]
    k0, k1 = slab_range(nz, rank, world)
    lo, hi = neighbours(cfg, rank, world)
    bc = [tuple(b) for b in cfg["bc"]]
    bc[2] = ("halo" if lo is not None else bc[2][0], "halo" if hi is not None else bc[2][1])
    x0 = list(cfg["x0"])
    x0[2] = cfg["x0"][2] + k0 * cfg["dx"][2]
    nx = list(cfg["nx"])
    nx[2] = k1 - k0
    return dict(cfg, nx=tuple(nx), x0=tuple(x0), bc=tuple(bc))


def slab_cells(cfg, rank, world):
    """Slice of the global cell index (cell-major, x1 fastest) owned by rank."""
    k0, k1 = slab_range(cfg["nx"][2], rank, world)
    P = cfg["nx"][0] * cfg["nx"][1]
    return slice(k0 * P, k1 * P)


def halo_fluid(cfg, fields, rank, world):
    """Fluid of the rank's ghost planes (two below, two above, wrapping a
    periodic x3), per side an array [2 * P, 7] of (rho, kappa, alpha_s
    coefficient, u^0, u^1, u^2, u^3), from the global per-cell fields."""
    import numpy as np
    nz = cfg["nx"][2]
    P = cfg["nx"][0] * cfg["nx"][1]
    k0, k1 = slab_range(nz, rank, world)
    cols = [np.asarray(fields[k], dtype=np.float64).reshape(nz, P, -1)
            for k in ("rho", "kappa", "alpha_s", "ucon")]
    out = []
    for planes in ((k0 - 2, k0 - 1), (k1, k1 + 1)):
        rows = []
        for k in planes:
            kk = min(max(k, 0), nz - 1) if cfg["bc"][2][0] != "periodic" else k % nz
            rows.append(np.concatenate([c[kk] for c in cols], axis=1))
        out.append(np.ascontiguousarray(np.concatenate(rows, axis=0)))
    return out[0], out[1]


class DistExchange:
    """Halo exchange with the x3 neighbours over torch.distributed
    point-to-point (isend/irecv): this rank's lo block goes to the lower
    neighbour (its upper ghost planes), the hi block to the upper one."""

    def __init__(self, cfg, rank, world, group=None):
        self.lo, self.hi = neighbours(cfg, rank, world)
        self.group = group

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        """Sends are posted lo then hi and receives hi then lo, and each block
        is tagged with the ghost side it fills (0 lower, 1 upper): with two
        ranks on a periodic ring both neighbours are the same rank, and the
        n-th receive from a rank must meet that rank's n-th send (NCCL matches
        point-to-point calls by order, gloo by tag)."""
        import torch.distributed as dist
        ops = []
        if self.lo is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, self.lo, self.group, tag=1))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, self.hi, self.group, tag=0))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, self.hi, self.group, tag=1))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, self.lo, self.group, tag=0))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


class SlabDriver:
    """Steps one slab through whole steps, exchanging its halo before every
    stage (two per step for order 2, one for order 1)."""

    def __init__(self, stepper, exchange, order=2):
        self.st = stepper
        self.ex = exchange
        self.nstage = 1 if order == 1 else 2

    def step(self, dt, nsteps):
        fails = 0
        for _ in range(nsteps):
            for stage in range(self.nstage):
                lo, hi = self.st.halo_pack(stage)
                rlo, rhi = self.st.halo_recv_buffers()
                self.ex.exchange(lo, hi, rlo, rhi)
                self.st.halo_unpack(rlo, rhi)
                fails += self.st.step_stage(dt, stage)
        return fails


class LocalExchange:
    """Every slab of the box in this process: step_all runs the stages of all
    slabs in lockstep, copying each slab's packs into its neighbours' ghost
    planes before every stage."""

    def __init__(self, cfg, steppers, order=2):
        self.cfg = cfg
        self.st = steppers
        self.world = len(steppers)
        self.nstage = 1 if order == 1 else 2

    def step_all(self, dt, nsteps):
        fails = 0
        for _ in range(nsteps):
            for stage in range(self.nstage):
                packs = [s.halo_pack(stage) for s in self.st]
                for r, s in enumerate(self.st):
                    lo, hi = neighbours(self.cfg, r, self.world)
                    rlo, rhi = s.halo_recv_buffers()
                    if lo is not None:
                        _copy(rlo, packs[lo][1])
                    if hi is not None:
                        _copy(rhi, packs[hi][0])
                    s.halo_unpack(rlo, rhi)
                for s in self.st:
                    fails += s.step_stage(dt, stage)
        return fails


def _copy(dst, src):
    if hasattr(dst, "copy_"):
        dst.copy_(src)
    else:
        dst[...] = src
