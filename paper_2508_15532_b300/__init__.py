"""B300-native radiation step of the covariant gray radiative transfer method
(Wallace, Begue & Pe'er; cuHARM radiation module).

Thin ctypes binding over the C ABI of ``include/rt.h`` (librt_b300.so):
argument marshalling only.  Every step of the computation runs in the CUDA
kernels of the library; there is no CPU fallback, and importing the binding
fails loudly when the library has not been built.

Arrays may be torch tensors (device or host) or numpy arrays (host); the
library copies with cudaMemcpyDefault on the context's stream.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt_b300.so")

RT_STATUS = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENOCONV", 5: "RT_ESTATE",
             6: "RT_ETIMEOUT"}
BC = {"periodic": 0, "outflow": 1, "pole": 2, "beam": 3, "halo": 4}
METRIC = {"minkowski": 0, "kerr_schild": 1, "snake": 2, "cart_cyl_tetrad": 3}
LIMITER = {"mc": 0, "minmod": 1, "donor": 2}
ANG = {"mapr": 0, "donor": 1}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}


class RTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (RT_STATUS.get(status, status), msg))
        self.status = status


class rt_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int * 3), ("x0", C.c_double * 3), ("dx", C.c_double * 3), ("bc", (C.c_int * 2) * 3),
        ("beam_dir", C.c_int), ("beam_lo", C.c_int), ("beam_hi", C.c_int), ("beam_I", C.c_double),
        ("n_pole_zero", C.c_int), ("gam", C.c_double), ("arad", C.c_double), ("rho_exp", C.c_double),
        ("T_exp", C.c_double), ("rho_floor", C.c_double), ("abar", C.c_double), ("tau_dt", C.c_int),
        ("order", C.c_int), ("limiter", C.c_int), ("ang_recon", C.c_int), ("transport", C.c_int),
        ("source", C.c_int), ("n0_cut", C.c_double), ("precision", C.c_int),
        ("coupling", C.c_int),
    ]


_lib = None
EXPORTS = ["rt_create_geodesic_grid", "rt_grid_query", "rt_destroy_grid", "rt_create", "rt_destroy",
           "rt_last_error", "rt_set_metric", "rt_set_fluid", "rt_set_intensity", "rt_get_intensity",
           "rt_set_ugas", "rt_get_ugas", "rt_cfl_dt", "rt_step", "rt_moments", "rt_grid_last_error",
           "rt_set_timing", "rt_get_timing", "rt_cfl_dt_noalloc", "rt_step_adjoint",
           "rt_step_record", "rt_step_adjoint_recorded"]


def lib():
    """Load librt_b300.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librt_b300.so is not built; run python -m paper_2508_15532_b300._build")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.rt_create_geodesic_grid.argtypes = [i, C.POINTER(vp)]
        L.rt_grid_query.argtypes = [vp, C.POINTER(i), C.POINTER(i), vp, vp]
        L.rt_destroy_grid.argtypes = [vp]
        L.rt_destroy_grid.restype = None
        L.rt_create.argtypes = [vp, C.POINTER(rt_config), vp, C.POINTER(vp)]
        L.rt_destroy.argtypes = [vp]
        L.rt_destroy.restype = None
        L.rt_last_error.argtypes = [vp]
        L.rt_last_error.restype = C.c_char_p
        L.rt_set_metric.argtypes = [vp, i, vp]
        L.rt_set_fluid.argtypes = [vp] * 7
        L.rt_set_intensity.argtypes = [vp, vp]
        L.rt_get_intensity.argtypes = [vp, vp]
        L.rt_set_ugas.argtypes = [vp, vp]
        L.rt_get_ugas.argtypes = [vp, vp]
        L.rt_cfl_dt.argtypes = [vp, d, C.POINTER(d)]
        L.rt_step.argtypes = [vp, d, i, C.POINTER(d), C.POINTER(C.c_longlong)]
        L.rt_moments.argtypes = [vp, vp, vp, vp]
        L.rt_grid_last_error.restype = C.c_char_p
        L.rt_set_timing.argtypes = [vp, i]
        L.rt_get_timing.argtypes = [vp, C.POINTER(d), C.POINTER(C.c_longlong)]
        L.rt_cfl_dt_noalloc.argtypes = [vp, d, C.POINTER(d)]
        L.rt_step_adjoint.argtypes = [vp, vp, vp, d, i, vp, vp, vp, vp, vp, vp]
        L.rt_step_record.argtypes = [vp, d, i, C.POINTER(d), C.POINTER(C.c_longlong)]
        L.rt_step_adjoint_recorded.argtypes = [vp, C.c_longlong, vp, vp, vp, vp, vp, vp]
        L.rt_step_stage.argtypes = [vp, d, i, C.POINTER(C.c_longlong)]
        L.rt_halo_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.rt_halo_pack.argtypes = [vp, i, vp, vp]
        L.rt_halo_unpack.argtypes = [vp, i, vp, vp]
        L.rt_set_fluid_halo.argtypes = [vp, vp, vp]
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a torch tensor or a C-contiguous numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch tensor or numpy array")


class Grid:
    """Geodesic angular grid (rt_create_geodesic_grid)."""

    def __init__(self, n):
        h = C.c_void_p()
        st = lib().rt_create_geodesic_grid(int(n), C.byref(h))
        if st:
            raise RTError(st, lib().rt_grid_last_error().decode())
        self.h = h
        nd, ne = C.c_int(), C.c_int()
        lib().rt_grid_query(h, C.byref(nd), C.byref(ne), None, None)
        self.nd, self.ne = nd.value, ne.value

    def query(self):
        d = np.zeros((self.nd, 3)); w = np.zeros(self.nd)
        lib().rt_grid_query(self.h, None, None, d.ctypes.data, w.ctypes.data)
        return d, w

    def __del__(self):
        if getattr(self, "h", None):
            lib().rt_destroy_grid(self.h)
            self.h = None


def make_config(cfg: dict, precision="fp64") -> rt_config:
    c = rt_config()
    for a in range(3):
        c.nx[a] = int(cfg["nx"][a]); c.x0[a] = float(cfg["x0"][a]); c.dx[a] = float(cfg["dx"][a])
        for s in range(2):
            c.bc[a][s] = BC[cfg["bc"][a][s]]
    c.beam_dir = int(cfg.get("beam_dir", -1)); c.beam_lo = int(cfg.get("beam_lo", 0))
    c.beam_hi = int(cfg.get("beam_hi", 0)); c.beam_I = float(cfg.get("beam_I", 0.0))
    c.n_pole_zero = int(cfg.get("n_pole_zero", 0))
    c.gam = float(cfg.get("gam", 5.0 / 3.0)); c.arad = float(cfg.get("arad", 1.0))
    c.rho_exp = float(cfg.get("rho_exp", 1.0)); c.T_exp = float(cfg.get("T_exp", 3.5))
    c.rho_floor = float(cfg.get("rho_floor", 5e-4)); c.abar = float(cfg.get("abar", 1.0))
    c.tau_dt = int(bool(cfg.get("tau_dt", False))); c.order = int(cfg.get("order", 2))
    c.limiter = LIMITER[cfg.get("limiter", "mc")]; c.ang_recon = ANG[cfg.get("ang_recon", "mapr")]
    c.transport = int(bool(cfg.get("transport", True))); c.source = int(bool(cfg.get("source", True)))
    c.n0_cut = float(cfg.get("n0_cut", 0.1)); c.precision = PRECISION[precision]
    c.coupling = int(cfg.get("coupling", 3))
    return c


class RadiationStep:
    """One problem on the current CUDA device (rt_create ... rt_destroy)."""

    def __init__(self, grid: Grid, cfg: dict, precision="fp64", stream=None):
        self.grid = grid
        self.cfg = dict(cfg)
        self.precision = precision
        self._c = make_config(cfg, precision)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        st = lib().rt_create(grid.h, C.byref(self._c), C.c_void_p(stream), C.byref(h))
        if st:
            raise RTError(st, lib().rt_last_error(None).decode())
        self.h = h
        self.fluid_token = None
        self.rec_id = 0
        self.nd = grid.nd
        self.ncell = int(np.prod(cfg["nx"]))
        coords = cfg.get("coords", "minkowski")
        params = ([cfg.get("snake_A", 0.0), cfg.get("snake_k", 0.0)] if coords == "snake"
                  else [cfg.get("M", 1.0), cfg.get("a", 0.0)])
        self._params = np.array(params, dtype=np.float64)
        self._check(lib().rt_set_metric(h, METRIC[coords], self._params.ctypes.data))

    def _check(self, st):
        if st:
            raise RTError(st, lib().rt_last_error(self.h).decode())

    def __del__(self):
        if getattr(self, "h", None):
            lib().rt_destroy(self.h)
            self.h = None

    def set_fluid(self, rho, ug, ucon, kappa, alpha_s, eta=None):
        self._keep = (rho, ug, ucon, kappa, alpha_s, eta)
        self.fluid_token = object()    # identifies this fluid (the library drops its recording)
        self.rec_id = 0
        self._check(lib().rt_set_fluid(self.h, _ptr(rho), _ptr(ug), _ptr(ucon), _ptr(kappa), _ptr(alpha_s), _ptr(eta)))

    def set_intensity(self, I):
        self._check(lib().rt_set_intensity(self.h, _ptr(I)))

    def get_intensity(self, out):
        self._check(lib().rt_get_intensity(self.h, _ptr(out)))
        return out

    def set_ugas(self, ug):
        self._check(lib().rt_set_ugas(self.h, _ptr(ug)))

    def get_ugas(self, out):
        self._check(lib().rt_get_ugas(self.h, _ptr(out)))
        return out

    def cfl_dt(self, cfl=0.4):
        d = C.c_double()
        self._check(lib().rt_cfl_dt(self.h, float(cfl), C.byref(d)))
        return d.value

    def cfl_dt_noalloc(self, cfl=0.4):
        """cfl_dt for callers that cannot allocate device memory between
        steps: the reduction runs in a fixed static scratch array inside the
        library (see rt_cfl_dt_noalloc)."""
        d = C.c_double()
        self._check(lib().rt_cfl_dt_noalloc(self.h, float(cfl), C.byref(d)))
        return d.value

    def step(self, dt, nsteps=1, check=False):
        used = C.c_double()
        nf = C.c_longlong()
        self._check(lib().rt_step(self.h, float(dt), int(nsteps), C.byref(used), C.byref(nf) if check else None))
        return used.value, (nf.value if check else None)

    def step_adjoint(self, I_ckpt, ug_ckpt, dt, nsteps, dL_dI_out, dL_dug_out, dL_dI_in, dL_dug_in,
                     dL_dkappa, dL_deta):
        """Reverse of nsteps steps from the checkpoint (rt_step_adjoint):
        writes dL_dI_in, dL_dug_in and adds to dL_dkappa, dL_deta."""
        self.rec_id = 0    # the recompute replaces any recording
        self._check(lib().rt_step_adjoint(self.h, _ptr(I_ckpt), _ptr(ug_ckpt), float(dt), int(nsteps),
                                          _ptr(dL_dI_out), _ptr(dL_dug_out), _ptr(dL_dI_in), _ptr(dL_dug_in),
                                          _ptr(dL_dkappa), _ptr(dL_deta)))

    def step_record(self, dt, nsteps):
        """nsteps steps as step(), keeping every stage's states for the
        reverse pass (rt_step_record); returns the recording's id."""
        used = C.c_double()
        rid = C.c_longlong()
        self.rec_id = 0
        self._check(lib().rt_step_record(self.h, float(dt), int(nsteps), C.byref(used), C.byref(rid)))
        self.rec_id = rid.value
        return rid.value

    def step_adjoint_recorded(self, rec_id, dL_dI_out, dL_dug_out, dL_dI_in, dL_dug_in, dL_dkappa, dL_deta):
        """Reverse of the recorded steps without their recompute
        (rt_step_adjoint_recorded)."""
        self._check(lib().rt_step_adjoint_recorded(self.h, int(rec_id), _ptr(dL_dI_out), _ptr(dL_dug_out),
                                                   _ptr(dL_dI_in), _ptr(dL_dug_in), _ptr(dL_dkappa), _ptr(dL_deta)))

    def set_timing(self, on=True):
        self._check(lib().rt_set_timing(self.h, int(bool(on))))

    def get_timing(self):
        """(summed stage-kernel device time in ms, launches) since the last call."""
        ms, n = C.c_double(), C.c_longlong()
        self._check(lib().rt_get_timing(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    # ---- x3 slab of a decomposed box (RT_BC_HALO faces; see partition.py)
    def step_stage(self, dt, stage, check=False):
        """One stage of a step (rt_step_stage); the unconverged solves if check."""
        nf = C.c_longlong()
        self._check(lib().rt_step_stage(self.h, float(dt), int(stage), C.byref(nf) if check else None))
        return nf.value if check else 0

    def halo_bytes(self):
        b = C.c_size_t()
        self._check(lib().rt_halo_bytes(self.h, C.byref(b)))
        return b.value

    def _halo_bufs(self):
        if getattr(self, "_hb", None) is None:
            import torch
            n = self.halo_bytes()
            self._hb = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(4)]
        return self._hb

    def halo_pack(self, stage):
        """(lo, hi) device byte tensors: the halo blocks of the source of
        `stage` (rt_halo_pack); reused by the next call."""
        b = self._halo_bufs()
        self._check(lib().rt_halo_pack(self.h, int(stage), _ptr(b[0]), _ptr(b[1])))
        self._pack_stage = int(stage)
        return b[0], b[1]

    def halo_recv_buffers(self):
        b = self._halo_bufs()
        return b[2], b[3]

    def halo_unpack(self, lo, hi, stage=None):
        stage = self._pack_stage if stage is None else stage
        self._check(lib().rt_halo_unpack(self.h, int(stage), _ptr(lo), _ptr(hi)))

    def set_fluid_halo(self, lo, hi):
        """Fluid of the ghost planes, per side [2 nx0 nx1, 7] float64 (rho,
        kappa, alpha_s coefficient, u^0..u^3)."""
        self._keep_halo = (lo, hi)
        self._check(lib().rt_set_fluid_halo(self.h, _ptr(lo), _ptr(hi)))

    def moments(self, R=None, Ebar=None, G=None):
        self._check(lib().rt_moments(self.h, _ptr(R), _ptr(Ebar), _ptr(G)))
        return R, Ebar, G
