"""ctypes binding of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load it; the product path never does.
The oracle shares no code with the CUDA library; both read the same config
dictionary (see ``paper_2508_15532_b300.workloads``).
"""
import ctypes as C

import numpy as np

from .build import build

BC = {"periodic": 0, "outflow": 1, "pole": 2, "beam": 3, "halo": 4}
COORDS = {"minkowski": 0, "kerr_schild": 1, "snake": 2, "cart_cyl_tetrad": 3}
LIMITER = {"mc": 0, "minmod": 1, "donor": 2}
ANG = {"mapr": 0, "donor": 1}


class _Cfg(C.Structure):
    _fields_ = [
        ("n_geo", C.c_int), ("nx", C.c_int * 3), ("x0", C.c_double * 3), ("dx", C.c_double * 3),
        ("coords", C.c_int), ("M", C.c_double), ("a", C.c_double), ("bc", (C.c_int * 2) * 3),
        ("beam_dir", C.c_int), ("beam_lo", C.c_int), ("beam_hi", C.c_int), ("beam_I", C.c_double),
        ("n_pole_zero", C.c_int), ("gam", C.c_double), ("arad", C.c_double),
        ("rho_exp", C.c_double), ("T_exp", C.c_double), ("rho_floor", C.c_double),
        ("abar", C.c_double), ("tau_dt", C.c_int), ("order", C.c_int), ("limiter", C.c_int),
        ("ang_recon", C.c_int), ("transport", C.c_int), ("source", C.c_int), ("n0_cut", C.c_double),
        ("coupling", C.c_int), ("snake_A", C.c_double), ("snake_k", C.c_double),
    ]


_libs = {}
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib(mutant: int = 0):
    """The oracle library; mutant > 0 loads a build with one planted mistake
    (only the test that shows the pins catch such mistakes asks for one)."""
    if mutant not in _libs:
        L = C.CDLL(build(mutant=mutant))
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Cfg)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_error.restype = C.c_char_p
        L.or_grid_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.or_grid_get.argtypes = [C.c_void_p, _D, _D, _I, _I, _I, _D, _D, _D]
        L.or_grid_mirror.argtypes = [C.c_void_p, _I]
        L.or_set_fluid.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D]
        L.or_set_intensity.argtypes = [C.c_void_p, _D]
        L.or_get_intensity.argtypes = [C.c_void_p, _D]
        L.or_get_ug.argtypes = [C.c_void_p, _D]
        L.or_set_ug.argtypes = [C.c_void_p, _D]
        L.or_cfl_dt.restype = C.c_double
        L.or_cfl_dt.argtypes = [C.c_void_p, C.c_double]
        L.or_step.restype = C.c_long
        L.or_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.or_step_stage.restype = C.c_long
        L.or_step_stage.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.or_halo_doubles.restype = C.c_size_t
        L.or_halo_doubles.argtypes = [C.c_void_p]
        L.or_halo_pack.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.or_halo_unpack.argtypes = [C.c_void_p, _D, _D]
        L.or_set_fluid_halo.argtypes = [C.c_void_p, _D, _D]
        L.or_source_only.restype = C.c_long
        L.or_source_only.argtypes = [C.c_void_p, C.c_double]
        L.or_moments.argtypes = [C.c_void_p, _D, _D, _D]
        L.or_geometry_at.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.or_edge_speeds.argtypes = [C.c_void_p, C.c_int, _D]
        L.or_face_flux.restype = C.c_double
        L.or_face_flux.argtypes = [C.c_double] * 8
        L.or_mapr.argtypes = [C.c_void_p, _D, _D]
        L.or_adjoint.argtypes = [C.c_void_p, _D, _D, C.c_int, C.c_double, _D, _D, _D, _D, _D]
        L.or_ghost_fill.argtypes = [C.c_void_p, _D, C.c_void_p, _I]
        _libs[mutant] = L
    return _libs[mutant]


def make_cfg(cfg: dict) -> _Cfg:
    c = _Cfg()
    c.n_geo = int(cfg["n_geo"])
    for a in range(3):
        c.nx[a] = int(cfg["nx"][a]); c.x0[a] = float(cfg["x0"][a]); c.dx[a] = float(cfg["dx"][a])
        for s in range(2):
            c.bc[a][s] = BC[cfg["bc"][a][s]]
    c.coords = COORDS[cfg.get("coords", "minkowski")]
    c.M = float(cfg.get("M", 1.0)); c.a = float(cfg.get("a", 0.0))
    c.beam_dir = int(cfg.get("beam_dir", -1)); c.beam_lo = int(cfg.get("beam_lo", 0))
    c.beam_hi = int(cfg.get("beam_hi", 0)); c.beam_I = float(cfg.get("beam_I", 0.0))
    c.n_pole_zero = int(cfg.get("n_pole_zero", 0))
    c.gam = float(cfg.get("gam", 5.0 / 3.0)); c.arad = float(cfg.get("arad", 1.0))
    c.rho_exp = float(cfg.get("rho_exp", 1.0)); c.T_exp = float(cfg.get("T_exp", 3.5))
    c.rho_floor = float(cfg.get("rho_floor", 5e-4)); c.abar = float(cfg.get("abar", 1.0))
    c.tau_dt = int(bool(cfg.get("tau_dt", False))); c.order = int(cfg.get("order", 2))
    c.limiter = LIMITER[cfg.get("limiter", "mc")]; c.ang_recon = ANG[cfg.get("ang_recon", "mapr")]
    c.transport = int(bool(cfg.get("transport", True))); c.source = int(bool(cfg.get("source", True)))
    c.n0_cut = float(cfg.get("n0_cut", 0.1))
    c.coupling = int(cfg.get("coupling", 3))
    c.snake_A = float(cfg.get("snake_A", 0.0)); c.snake_k = float(cfg.get("snake_k", 0.0))
    return c


def _f(x):
    return np.ascontiguousarray(x, dtype=np.float64).ravel()


class Oracle:
    """One oracle problem: grid, geometry, fluid and intensity state."""

    def __init__(self, cfg: dict, mutant: int = 0):
        self.cfg = dict(cfg)
        self._c = make_cfg(cfg)
        self.L = lib(mutant)
        self.h = self.L.or_create(C.byref(self._c))
        if not self.h:
            raise RuntimeError("oracle: " + self.L.or_error().decode())
        nd, ne = C.c_int(), C.c_int()
        self.L.or_grid_sizes(self.h, C.byref(nd), C.byref(ne))
        self.nd, self.ne = nd.value, ne.value
        self.ncell = int(np.prod(cfg["nx"]))

    def __del__(self):
        if getattr(self, "h", None):
            self.L.or_destroy(self.h)
            self.h = None

    def grid(self):
        nd, ne = self.nd, self.ne
        d = dict(dir=np.zeros((nd, 3)), w=np.zeros(nd), nnb=np.zeros(nd, np.int32),
                 nbr=np.zeros((nd, 6), np.int32), edge=np.zeros((ne, 2), np.int32),
                 dlam=np.zeros(ne), emid=np.zeros((ne, 3)), eu=np.zeros((ne, 3)))
        self.L.or_grid_get(self.h, d["dir"], d["w"], d["nnb"], d["nbr"], d["edge"], d["dlam"], d["emid"], d["eu"])
        m = np.zeros(nd, np.int32)
        self.L.or_grid_mirror(self.h, m)
        d["mirror"] = m
        return d

    def set_fluid(self, rho, ug, ucon, kappa, alpha_s, eta=None):
        eta = np.ones(self.ncell) if eta is None else eta
        self.L.or_set_fluid(self.h, _f(rho), _f(ug), _f(ucon), _f(kappa), _f(alpha_s), _f(eta))

    def set_intensity(self, I):
        self.L.or_set_intensity(self.h, _f(I))

    def set_ug(self, ug):
        self.L.or_set_ug(self.h, _f(ug))

    def intensity(self):
        out = np.zeros(self.ncell * self.nd)
        self.L.or_get_intensity(self.h, out)
        return out.reshape(self.ncell, self.nd)

    def ug(self):
        out = np.zeros(self.ncell)
        self.L.or_get_ug(self.h, out)
        return out

    def cfl_dt(self, cfl):
        return self.L.or_cfl_dt(self.h, float(cfl))

    def step_stage(self, dt, stage):
        """One stage of a step (0: predictor or the single Euler stage, 1:
        corrector); the unconverged temperature solves of the stage."""
        r = self.L.or_step_stage(self.h, float(dt), int(stage))
        if r < 0:
            raise RuntimeError("oracle: " + self.L.or_error().decode())
        return r

    def halo_doubles(self):
        return int(self.L.or_halo_doubles(self.h))

    def halo_pack(self, stage):
        """(lo, hi): the first and last two owned x3 planes of the source of
        `stage` (intensities, then gas energies)."""
        n = self.halo_doubles()
        lo, hi = np.empty(n), np.empty(n)
        if self.L.or_halo_pack(self.h, int(stage), lo, hi):
            raise RuntimeError("oracle: " + self.L.or_error().decode())
        return lo, hi

    def halo_unpack(self, lo, hi):
        if self.L.or_halo_unpack(self.h, _f(lo), _f(hi)):
            raise RuntimeError("oracle: " + self.L.or_error().decode())

    def set_fluid_halo(self, lo, hi):
        """Fluid of the ghost planes, per side [2 planes * P, 7] as (rho,
        kappa, alpha_s coefficient, u^0..u^3)."""
        if self.L.or_set_fluid_halo(self.h, _f(lo), _f(hi)):
            raise RuntimeError("oracle: " + self.L.or_error().decode())

    def step(self, dt, nsteps=1):
        return self.L.or_step(self.h, float(dt), int(nsteps))

    def source_only(self, dt):
        return self.L.or_source_only(self.h, float(dt))

    def moments(self):
        R = np.zeros(self.ncell * 10); E = np.zeros(self.ncell); G = np.zeros(self.ncell * 4)
        self.L.or_moments(self.h, R, E, G)
        return R.reshape(-1, 10), E, G.reshape(-1, 4)

    def geometry_at(self, x):
        g = np.zeros(16); e = np.zeros(16); om = np.zeros(64); sg = np.zeros(1)
        self.L.or_geometry_at(self.h, _f(x), g, e, om, sg)
        return g.reshape(4, 4), e.reshape(4, 4), om.reshape(4, 4, 4), sg[0]

    def edge_speeds(self, cell):
        w = np.zeros(self.ne)
        self.L.or_edge_speeds(self.h, int(cell), w)
        return w

    def mapr(self, Icell):
        out = np.zeros(self.nd * 6)
        self.L.or_mapr(self.h, _f(Icell), out)
        return out.reshape(self.nd, 6)

    def ghosts(self, I):
        """The ghosted copy of I the transport stage reads, shape (gn2, gn1, gn0, nd)."""
        gn = np.zeros(3, np.int32)
        self.L.or_ghost_fill(self.h, _f(I), None, gn)
        out = np.zeros(int(np.prod(gn)) * self.nd)
        self.L.or_ghost_fill(self.h, _f(I), out.ctypes.data_as(C.c_void_p), gn)
        return out.reshape(gn[2], gn[1], gn[0], self.nd)

    def adjoint(self, I0, ug0, nsteps, dt, dL_dI, dL_dug):
        gI = np.zeros(self.ncell * self.nd); gk = np.zeros(self.ncell); ge = np.zeros(self.ncell)
        rc = self.L.or_adjoint(self.h, _f(I0), _f(ug0), int(nsteps), float(dt), _f(dL_dI), _f(dL_dug), gI, gk, ge)
        if rc != 0:
            raise RuntimeError("oracle adjoint: " + self.L.or_error().decode())
        return gI.reshape(self.ncell, self.nd), gk, ge


def face_flux(n, IL, IR, Il, Ir, tau, vL=0.0, vR=0.0):
    return lib().or_face_flux(float(n), float(IL), float(IR), float(Il), float(Ir), float(tau), float(vL), float(vR))
