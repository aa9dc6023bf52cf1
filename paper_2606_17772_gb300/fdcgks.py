"""Python binding of libfdcgks.so (ctypes; argument marshalling only).

Every step of the FD-CGKS path runs in the library's CUDA kernels; this module
only passes pointers, sizes and the current torch CUDA stream across the C
ABI declared in include/fdcgks.h.  There is no fallback: if the library is
missing or the GPU is unavailable, the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

BC_PERIODIC, BC_TRANSMISSIVE, BC_SYMMETRY, BC_NOSLIP, BC_FIXED = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "non-physical state", 4: "no state loaded",
          5: "device wait timed out", 6: "out of device memory"}

EXPORTS = ["fdcgks_create", "fdcgks_destroy", "fdcgks_dims", "fdcgks_set_state", "fdcgks_get_state",
           "fdcgks_step", "fdcgks_steps", "fdcgks_cfl_dt", "fdcgks_cfl_dt_sum", "fdcgks_check", "fdcgks_stage_operator",
           "fdcgks_iface_batch", "fdcgks_nodal_batch", "fdcgks_recon_batch", "fdcgks_last_error",
           "fdcgks_status_string", "fdcgks_set_profiling", "fdcgks_get_profile", "fdcgks_cfl_dt_noalloc",
           "fdcgks_ens_create", "fdcgks_ens_destroy", "fdcgks_ens_set_state", "fdcgks_ens_get_state",
           "fdcgks_ens_run", "fdcgks_ens_status", "fdcgks_ens_set_tiles", "fdcgks_ens_get_tiles",
           "fdcgks_ens_tune", "fdcgks_ens_profile", "fdcgks_ens_info", "fdcgks_ens_last_error",
           "fdcgks_vjp_steps", "fdcgks_set_sides", "fdcgks_set_time", "fdcgks_get_time",
           "fdcgks_line_create", "fdcgks_line_destroy", "fdcgks_line_set_state", "fdcgks_line_get_state",
           "fdcgks_line_steps", "fdcgks_line_run", "fdcgks_line_stage_operator", "fdcgks_line_check",
           "fdcgks_line_last_error"]

ENS_NONPHYSICAL, ENS_NO_WAVE_SPEED, ENS_FROZEN = 1, 2, 4


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("flux_variant", ctypes.c_int),
        ("geno_variant", ctypes.c_int),
        ("grad_base", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("tau_c1", ctypes.c_double), ("tau_c2", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("recon_vars", ctypes.c_int),
    ]


class LineParams(ctypes.Structure):
    """fdcgks_line_params: a batch of lines of the one-dimensional scheme."""
    _fields_ = [
        ("n", ctypes.c_int), ("batch", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
        ("bc", ctypes.c_int * 2),
        ("flux_variant", ctypes.c_int), ("geno_variant", ctypes.c_int), ("grad_base", ctypes.c_int),
        ("tau_c1", ctypes.c_double), ("tau_c2", ctypes.c_double),
        ("recon_vars", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("cluster", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


def line_params(n, batch=1, x0=0.0, x1=1.0, gamma=1.4, mu=0.0, Pr=1.0, bc=(1, 1), flux_variant=64,
                geno_variant=0, grad_base=0, tau_c1=0.0, tau_c2=0.0, recon_vars=0, stream=None, cluster=0,
                precision=FP64):
    p = LineParams()
    p.n, p.batch, p.x0, p.x1 = n, batch, x0, x1
    p.gamma, p.mu, p.Pr = gamma, mu, Pr
    p.bc[0], p.bc[1] = bc
    p.flux_variant, p.geno_variant, p.grad_base = flux_variant, geno_variant, grad_base
    p.tau_c1, p.tau_c2, p.recon_vars = tau_c1, tau_c2, recon_vars
    p.stream = stream
    p.cluster = cluster
    p.precision = precision
    return p


def line_params_for_case(case, batch=1, stream=None, cluster=0, precision=FP64):
    """LineParams of a strip case (inputs.Case; its x extent, gas, x-ends and options)."""
    return line_params(case.nx, batch, case.x0, case.x1, case.gamma, case.mu, case.Pr, tuple(case.bc[:2]),
                       case.flux_variant, case.geno_variant, case.grad_base, case.tau_c1, case.tau_c2,
                       case.recon_vars, stream, cluster, precision)


class Side(ctypes.Structure):
    """One boundary side split at split0 + split_speed * t (fdcgks_side)."""
    _fields_ = [
        ("kind", ctypes.c_int * 2),
        ("split0", ctypes.c_double), ("split_speed", ctypes.c_double),
        ("prim", (ctypes.c_double * 4) * 2),
    ]


def make_sides(sides):
    """Four fdcgks_side structs from a sequence of 4 dicts with keys kind
    (2 ints), split0, split_speed (default 0) and prim (2 x 4 floats, default
    zeros)."""
    arr = (Side * 4)()
    for k, sd in enumerate(sides):
        arr[k].kind[0], arr[k].kind[1] = sd["kind"]
        arr[k].split0 = sd.get("split0", 0.0)
        arr[k].split_speed = sd.get("split_speed", 0.0)
        prim = sd.get("prim", ((0.0,) * 4,) * 2)
        for q in range(2):
            for j in range(4):
                arr[k].prim[q][j] = prim[q][j]
    return arr


class FdcgksError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status


_lib = None
_VP = ctypes.c_void_p


def library_path():
    return _build.LIB


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise FileNotFoundError("libfdcgks.so not found at %s: build it with "
                                "paper_2606_17772_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    lib.fdcgks_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_VP)]
    lib.fdcgks_destroy.argtypes = [_VP]
    lib.fdcgks_destroy.restype = None
    lib.fdcgks_dims.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int)] * 4
    lib.fdcgks_set_state.argtypes = [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_get_state.argtypes = [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_step.argtypes = [_VP, ctypes.c_double]
    lib.fdcgks_steps.argtypes = [_VP, ctypes.c_double, ctypes.c_int]
    lib.fdcgks_cfl_dt.argtypes = [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.fdcgks_cfl_dt_sum.argtypes = [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.fdcgks_check.argtypes = [_VP, ctypes.POINTER(ctypes.c_int)]
    lib.fdcgks_stage_operator.argtypes = [_VP, ctypes.c_double] + [_VP] * 8
    lib.fdcgks_iface_batch.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double, ctypes.c_int, _VP, _VP]
    lib.fdcgks_nodal_batch.argtypes = [ctypes.POINTER(Params), ctypes.c_double, ctypes.c_int, _VP, _VP]
    lib.fdcgks_recon_batch.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_double, ctypes.c_int, _VP, _VP]
    lib.fdcgks_set_profiling.argtypes = [_VP, ctypes.c_int]
    lib.fdcgks_get_profile.argtypes = [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_longlong)]
    lib.fdcgks_cfl_dt_noalloc.argtypes = [ctypes.POINTER(Params), _VP, _VP, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double)]
    lib.fdcgks_ens_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(_VP)]
    lib.fdcgks_ens_destroy.argtypes = [_VP]
    lib.fdcgks_ens_destroy.restype = None
    lib.fdcgks_ens_set_state.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_ens_get_state.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_ens_run.argtypes = [_VP, ctypes.c_double, _VP, ctypes.c_int]
    lib.fdcgks_ens_status.argtypes = [_VP, _VP, _VP, _VP]
    lib.fdcgks_ens_set_tiles.argtypes = [_VP, _VP]
    lib.fdcgks_ens_get_tiles.argtypes = [_VP, _VP]
    lib.fdcgks_ens_tune.argtypes = [_VP, ctypes.c_double, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)]
    lib.fdcgks_ens_profile.argtypes = [_VP, ctypes.c_double, ctypes.c_int, _VP]
    lib.fdcgks_ens_info.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong)]
    lib.fdcgks_vjp_steps.argtypes = [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int] + [_VP] * 12
    lib.fdcgks_set_sides.argtypes = [_VP, _VP]
    lib.fdcgks_set_time.argtypes = [_VP, ctypes.c_double]
    lib.fdcgks_get_time.argtypes = [_VP, ctypes.POINTER(ctypes.c_double)]
    lib.fdcgks_line_create.argtypes = [ctypes.POINTER(LineParams), ctypes.POINTER(_VP)]
    lib.fdcgks_line_destroy.argtypes = [_VP]
    lib.fdcgks_line_destroy.restype = None
    lib.fdcgks_line_set_state.argtypes = [_VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_line_get_state.argtypes = [_VP, _VP, _VP, ctypes.c_int]
    lib.fdcgks_line_steps.argtypes = [_VP, ctypes.c_double, ctypes.c_int]
    lib.fdcgks_line_run.argtypes = [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int, _VP, _VP]
    lib.fdcgks_line_stage_operator.argtypes = [_VP, ctypes.c_double, _VP, _VP, _VP, _VP]
    lib.fdcgks_line_check.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int)]
    lib.fdcgks_line_last_error.argtypes = [_VP]
    lib.fdcgks_line_last_error.restype = ctypes.c_char_p
    lib.fdcgks_ens_last_error.argtypes = [_VP]
    lib.fdcgks_ens_last_error.restype = ctypes.c_char_p
    lib.fdcgks_last_error.argtypes = [_VP]
    lib.fdcgks_last_error.restype = ctypes.c_char_p
    lib.fdcgks_status_string.argtypes = [ctypes.c_int]
    lib.fdcgks_status_string.restype = ctypes.c_char_p
    for name in ("fdcgks_create", "fdcgks_dims", "fdcgks_set_state", "fdcgks_get_state", "fdcgks_step",
                 "fdcgks_steps", "fdcgks_cfl_dt", "fdcgks_cfl_dt_sum", "fdcgks_check", "fdcgks_stage_operator",
                 "fdcgks_iface_batch",
                 "fdcgks_nodal_batch", "fdcgks_recon_batch", "fdcgks_set_profiling", "fdcgks_get_profile",
                 "fdcgks_cfl_dt_noalloc", "fdcgks_ens_create", "fdcgks_ens_set_state", "fdcgks_ens_get_state",
                 "fdcgks_ens_run", "fdcgks_ens_status", "fdcgks_ens_set_tiles", "fdcgks_ens_get_tiles",
                 "fdcgks_ens_tune", "fdcgks_ens_profile", "fdcgks_ens_info", "fdcgks_vjp_steps",
                 "fdcgks_set_sides", "fdcgks_set_time", "fdcgks_get_time", "fdcgks_line_create",
                 "fdcgks_line_set_state", "fdcgks_line_get_state", "fdcgks_line_steps", "fdcgks_line_run",
                 "fdcgks_line_stage_operator", "fdcgks_line_check"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != 0:
        msg = load().fdcgks_last_error(ctx).decode()
        raise FdcgksError(status, msg)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _on_current_stream(params):
    """A copy of params whose stream is torch's current stream where the caller
    left it unset; the caller's own params object is not modified."""
    p = type(params).from_buffer_copy(params)
    if p.stream is None:
        p.stream = _stream().value
    return p


def make_params(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, mu=0.0, Pr=1.0, bc=(0, 0, 0, 0),
                flux_variant=64, geno_variant=0, grad_base=0, precision=FP64, tau_c1=0.0, tau_c2=0.0,
                stream=None, recon_vars=0):
    p = Params()
    p.nx, p.ny = nx, ny
    p.x0, p.x1, p.y0, p.y1 = x0, x1, y0, y1
    p.gamma, p.mu, p.Pr = gamma, mu, Pr
    for k in range(4):
        p.bc[k] = bc[k]
    p.flux_variant, p.geno_variant, p.grad_base = flux_variant, geno_variant, grad_base
    p.precision = precision
    p.tau_c1, p.tau_c2 = tau_c1, tau_c2
    p.stream = stream
    p.recon_vars = recon_vars
    return p


def params_for_case(case, precision=FP64, stream=None):
    """Params from a paper_2606_17772_gb300.inputs.Case (its split sides, if
    any, go through Solver.set_sides, which Solver.from_case calls)."""
    kw = case.oracle_kwargs()
    kw.pop("sides", None)
    return make_params(precision=precision, stream=stream, **kw)


def _dptr(t, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError("tensor has %d elements, expected %d" % (t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, numel=None):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        if numel is not None and a.size != numel:
            raise ValueError("array has %d elements, expected %d" % (a.size, numel))
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda:
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        if numel is not None and a.numel() != numel:
            raise ValueError("tensor has %d elements, expected %d" % (a.numel(), numel))
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a host array")


class Solver:
    """One FD-CGKS context (fdcgks_create ... fdcgks_destroy)."""

    def __init__(self, params):
        lib = load()
        params = _on_current_stream(params)
        self._p = params
        h = _VP()
        _check(lib.fdcgks_create(ctypes.byref(params), ctypes.byref(h)))
        self._h = h
        d = [ctypes.c_int() for _ in range(4)]
        _check(lib.fdcgks_dims(h, *[ctypes.byref(x) for x in d]), h)
        self.nx, self.ny, self.nxd, self.nyd = (x.value for x in d)

    @classmethod
    def from_case(cls, case, precision=FP64):
        s = cls(params_for_case(case, precision))
        if getattr(case, "sides", None) is not None:
            s.set_sides(case.sides)
        return s

    def set_sides(self, sides):
        """Split boundary sides (see make_sides); None restores params.bc."""
        arr = None if sides is None else make_sides(sides)
        _check(load().fdcgks_set_sides(self._h, arr), self._h)

    def set_time(self, t):
        _check(load().fdcgks_set_time(self._h, ctypes.c_double(t)), self._h)

    def get_time(self):
        out = ctypes.c_double()
        _check(load().fdcgks_get_time(self._h, ctypes.byref(out)), self._h)
        return out.value

    def close(self):
        if getattr(self, "_h", None):
            load().fdcgks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- sizes of the state arrays
    def shapes(self):
        return ((4, self.ny, self.nx), (2, 4, self.ny, self.nx), (4, self.nyd, self.nxd), (2, 4, self.nyd, self.nxd))

    def _ptrs(self, arrs, on_device):
        sizes = [int(np.prod(s)) for s in self.shapes()]
        conv = _dptr if on_device else _hptr
        return [conv(a, n) for a, n in zip(arrs, sizes)]

    def set_state(self, Wp, Gp, Wd, Gd):
        """Device (CUDA float64 tensors) or host (numpy / CPU tensors) arrays."""
        import torch
        on_device = isinstance(Wp, torch.Tensor) and Wp.is_cuda
        _check(load().fdcgks_set_state(self._h, *self._ptrs((Wp, Gp, Wd, Gd), on_device), int(on_device)), self._h)

    def get_state(self, out=None, device=True):
        import torch
        if out is None:
            if device:
                out = [torch.empty(s, dtype=torch.float64, device="cuda") for s in self.shapes()]
            else:
                out = [np.empty(s) for s in self.shapes()]
        on_device = isinstance(out[0], torch.Tensor) and out[0].is_cuda
        _check(load().fdcgks_get_state(self._h, *self._ptrs(out, on_device), int(on_device)), self._h)
        return tuple(out)

    def step(self, dt):
        _check(load().fdcgks_step(self._h, ctypes.c_double(dt)), self._h)

    def steps(self, dt, n):
        _check(load().fdcgks_steps(self._h, ctypes.c_double(dt), int(n)), self._h)

    def cfl_dt(self, cfl, form="direction"):
        """CFL time step: form "direction" (fdcgks_cfl_dt) or "sum" (fdcgks_cfl_dt_sum)."""
        out = ctypes.c_double()
        fn = load().fdcgks_cfl_dt_sum if form == "sum" else load().fdcgks_cfl_dt
        _check(fn(self._h, ctypes.c_double(cfl), ctypes.byref(out)), self._h)
        return out.value

    def check(self):
        out = ctypes.c_int()
        _check(load().fdcgks_check(self._h, ctypes.byref(out)), self._h)
        return bool(out.value)

    def set_profiling(self, enable=True):
        _check(load().fdcgks_set_profiling(self._h, int(bool(enable))), self._h)

    def get_profile(self):
        """(ms per class, launch groups per class, total launches); classes: ghost, nodal, points, update, cfl."""
        ms = (ctypes.c_double * 5)()
        cn = (ctypes.c_int * 5)()
        n = ctypes.c_longlong()
        _check(load().fdcgks_get_profile(self._h, ms, cn, ctypes.byref(n)), self._h)
        names = ("ghost", "nodal", "points", "update", "cfl")
        return dict(zip(names, list(ms))), dict(zip(names, list(cn))), n.value

    def launches(self):
        return self.get_profile()[2]

    def vjp_steps(self, dt, nsteps, state0, adj_final, checkpoint_every=50):
        """dJ/d(initial state) for dJ/d(final state) `adj_final` after `nsteps`
        steps of size dt from `state0` (both 4-tuples of CUDA float64 tensors in
        the set_state layouts).  The solver keeps the final state.  On a
        mixed-precision solver the trajectory is its own mixed run and the
        reverse pass is the FP64 step's along it."""
        import torch
        torch.cuda.current_stream().synchronize()
        out = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in self.shapes()]
        sizes = [int(np.prod(s)) for s in self.shapes()]
        ptrs = ([_dptr(a, n) for a, n in zip(state0, sizes)] + [_dptr(a, n) for a, n in zip(adj_final, sizes)] +
                [_dptr(a, n) for a, n in zip(out, sizes)])
        _check(load().fdcgks_vjp_steps(self._h, ctypes.c_double(dt), int(nsteps), int(checkpoint_every), *ptrs),
               self._h)
        return tuple(out)

    def stage_operator(self, dt):
        import torch
        sp, sg, sdp, sdg = self.shapes()
        out = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in
               [("Lp", sp), ("Ltp", sp), ("gbp", sg), ("gtp", sg), ("Ld", sdp), ("Ltd", sdp), ("gbd", sdg),
                ("gtd", sdg)]}
        ptrs = [_dptr(out[k]) for k in ("Lp", "Ltp", "gbp", "gtp", "Ld", "Ltd", "gbd", "gtd")]
        _check(load().fdcgks_stage_operator(self._h, ctypes.c_double(dt), *ptrs), self._h)
        return out


def iface_batch(params, normal, dt, inp, out=None):
    """Batched interface solves: inp [n, 20] CUDA float64 -> out [n, 24]."""
    import torch
    n = inp.shape[0]
    if out is None:
        out = torch.empty((n, 24), dtype=torch.float64, device=inp.device)
    params = _on_current_stream(params)
    _check(load().fdcgks_iface_batch(ctypes.byref(params), int(normal), ctypes.c_double(dt), n,
                                     _dptr(inp, 20 * n), _dptr(out, 24 * n)))
    return out


def nodal_batch(params, dt, inp, out=None):
    """Batched nodal fluxes: inp [n, 12] -> out [n, 16] (CUDA float64)."""
    import torch
    n = inp.shape[0]
    if out is None:
        out = torch.empty((n, 16), dtype=torch.float64, device=inp.device)
    params = _on_current_stream(params)
    _check(load().fdcgks_nodal_batch(ctypes.byref(params), ctypes.c_double(dt), n, _dptr(inp, 12 * n),
                                     _dptr(out, 16 * n)))
    return out


def recon_batch(params, kind, h, inp, out=None):
    """Batched GENO reconstructions: kind 0 inp [n, 8], kind 1 inp [n, 6] -> out [n, 6]."""
    import torch
    n = inp.shape[0]
    if out is None:
        out = torch.empty((n, 6), dtype=torch.float64, device=inp.device)
    params = _on_current_stream(params)
    _check(load().fdcgks_recon_batch(ctypes.byref(params), int(kind), ctypes.c_double(h), n,
                                     _dptr(inp, (8 if kind == 0 else 6) * n), _dptr(out, 6 * n)))
    return out


def cfl_dt_noalloc(params, Wp, Wd, cfl):
    """CFL time step from caller-owned device arrays without any allocation.

    For callers that cannot allocate device memory when they need a time step:
    an application that hands this library a fixed share of the GPU's memory
    and forbids further allocations, or a time loop that must not risk an
    allocation failure or the synchronisation that cudaMalloc and cudaFree can
    cause.  Wp: [4, ny, nx], Wd: [4, nyd, nxd] contiguous float64 CUDA
    tensors.  The call synchronizes the stream to return dt to the host.  The
    library keeps the partial maxima in a fixed device array shared by all
    calls; calls that overlap on the GPU race on it.  The first call on a
    device looks up that array's address, so make it before any stream
    capture.  params is not modified (an unset stream means torch's current
    stream for this call).
    """
    params = _on_current_stream(params)
    nxd = params.nx + (0 if params.bc[0] == BC_PERIODIC else 1)
    nyd = params.ny + (0 if params.bc[2] == BC_PERIODIC else 1)
    out = ctypes.c_double()
    _check(load().fdcgks_cfl_dt_noalloc(ctypes.byref(params), _dptr(Wp, 4 * params.nx * params.ny),
                                        _dptr(Wd, 4 * nxd * nyd), ctypes.c_double(cfl), ctypes.byref(out)))
    return out.value


def _echeck(status, ens):
    if status != 0:
        raise FdcgksError(status, load().fdcgks_ens_last_error(ens).decode())


class Ensemble:
    """A batch of independent runs advanced together (fdcgks_ens_create ... fdcgks_ens_destroy).

    members: a list of Params (one per run; all with the same precision).
    The ensemble works on its own CUDA stream (`stream`); every method but
    run() synchronizes it before returning.
    """

    def __init__(self, members):
        lib = load()
        self.count = len(members)
        arr = (Params * self.count)(*members)
        h = _VP()
        _check(lib.fdcgks_ens_create(arr, self.count, ctypes.byref(h)))
        self._h = h
        self.dims = []
        for p in members:
            nxd = p.nx + (0 if p.bc[0] == BC_PERIODIC else 1)
            nyd = p.ny + (0 if p.bc[2] == BC_PERIODIC else 1)
            self.dims.append((p.nx, p.ny, nxd, nyd))
        st, n = _VP(), ctypes.c_longlong()
        _echeck(lib.fdcgks_ens_info(h, ctypes.byref(st), None, ctypes.byref(n)), h)
        self.stream = st.value
        self.nodes = n.value

    @classmethod
    def from_cases(cls, cases, precision=FP64):
        if any(getattr(c, "sides", None) is not None for c in cases):
            raise ValueError("ensemble members take the boundary kinds of params.bc only (no split sides)")
        return cls([params_for_case(c, precision) for c in cases])

    def close(self):
        if getattr(self, "_h", None):
            load().fdcgks_ens_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def shapes(self, m):
        if not 0 <= m < self.count:
            raise IndexError("member %d out of range [0, %d)" % (m, self.count))
        nx, ny, nxd, nyd = self.dims[m]
        return ((4, ny, nx), (2, 4, ny, nx), (4, nyd, nxd), (2, 4, nyd, nxd))

    def _ptrs(self, m, arrs, on_device):
        sizes = [int(np.prod(s)) for s in self.shapes(m)]
        conv = _dptr if on_device else _hptr
        return [conv(a, n) for a, n in zip(arrs, sizes)]

    def set_state(self, m, Wp, Gp, Wd, Gd):
        import torch
        on_device = isinstance(Wp, torch.Tensor) and Wp.is_cuda
        if on_device:
            torch.cuda.current_stream().synchronize()
        _echeck(load().fdcgks_ens_set_state(self._h, int(m), *self._ptrs(m, (Wp, Gp, Wd, Gd), on_device),
                                            int(on_device)), self._h)

    def get_state(self, m, out=None, device=True):
        import torch
        if out is None:
            if device:
                out = [torch.empty(s, dtype=torch.float64, device="cuda") for s in self.shapes(m)]
            else:
                out = [np.empty(s) for s in self.shapes(m)]
        on_device = isinstance(out[0], torch.Tensor) and out[0].is_cuda
        _echeck(load().fdcgks_ens_get_state(self._h, int(m), *self._ptrs(m, out, on_device), int(on_device)),
                self._h)
        return tuple(out)

    def run(self, nsteps, cfl=0.4, dt=None):
        """nsteps steps; dt None: per-member CFL steps (cfl), else a sequence of fixed per-member steps."""
        if dt is None:
            ptr = None
        else:
            arr = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.count,)))
            ptr = ctypes.c_void_p(arr.ctypes.data)
        _echeck(load().fdcgks_ens_run(self._h, ctypes.c_double(cfl), ptr, int(nsteps)), self._h)

    def status(self):
        """(time since set_state, last dt, status bits) per member as numpy arrays."""
        t = np.zeros(self.count)
        d = np.zeros(self.count)
        s = np.zeros(self.count, dtype=np.int32)
        _echeck(load().fdcgks_ens_status(self._h, ctypes.c_void_p(t.ctypes.data), ctypes.c_void_p(d.ctypes.data),
                                         ctypes.c_void_p(s.ctypes.data)), self._h)
        return t, d, s

    def set_tiles(self, cfg):
        a = (ctypes.c_int * 4)(*cfg)
        _echeck(load().fdcgks_ens_set_tiles(self._h, a), self._h)

    def get_tiles(self):
        a = (ctypes.c_int * 4)()
        _echeck(load().fdcgks_ens_get_tiles(self._h, a), self._h)
        return list(a)

    def tune(self, cfl=0.4, trial_steps=3):
        """Autotune the tile configuration; returns (cfg, ms per step)."""
        a = (ctypes.c_int * 4)()
        ms = ctypes.c_double()
        _echeck(load().fdcgks_ens_tune(self._h, ctypes.c_double(cfl), int(trial_steps), a, ctypes.byref(ms)),
                self._h)
        return list(a), ms.value

    def profile(self, nsteps, cfl=0.4):
        """Advance nsteps CFL steps outside the graph; ms per phase (cfl, ghost, nodal, points, update)."""
        a = (ctypes.c_double * 5)()
        _echeck(load().fdcgks_ens_profile(self._h, ctypes.c_double(cfl), int(nsteps), a), self._h)
        return dict(zip(("cfl", "ghost", "nodal", "points", "update"), list(a)))

    def launches(self):
        n = ctypes.c_longlong()
        _echeck(load().fdcgks_ens_info(self._h, None, ctypes.byref(n), None), self._h)
        return n.value

    def synchronize(self):
        import torch
        torch.cuda.ExternalStream(self.stream).synchronize()


def _lcheck(status, lines):
    if status != 0:
        raise FdcgksError(status, load().fdcgks_line_last_error(lines).decode())


class Lines:
    """A batch of lines of the one-dimensional scheme (fdcgks_line_*).
    State arrays: W [batch][3][n] (rho, rho U, rho E) and Wx [batch][3][n]."""

    def __init__(self, params):
        lib = load()
        params = _on_current_stream(params)
        self._p = params
        h = _VP()
        _lcheck(lib.fdcgks_line_create(ctypes.byref(params), ctypes.byref(h)), None)
        self._h = h
        self.n, self.batch = params.n, params.batch

    @classmethod
    def from_case(cls, case, batch=1, cluster=0, precision=FP64):
        return cls(line_params_for_case(case, batch, cluster=cluster, precision=precision))

    def close(self):
        if getattr(self, "_h", None):
            load().fdcgks_line_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def shape(self):
        return (self.batch, 3, self.n)

    def set_state(self, W, Wx):
        """CUDA float64 tensors or host arrays of shape (batch, 3, n) (or (3, n) for one line)."""
        import torch
        on_device = isinstance(W, torch.Tensor) and W.is_cuda
        n = self.batch * 3 * self.n
        conv = _dptr if on_device else _hptr
        _lcheck(load().fdcgks_line_set_state(self._h, conv(W, n), conv(Wx, n), int(on_device)), self._h)

    def get_state(self, device=True):
        import torch
        if device:
            out = [torch.empty(self.shape(), dtype=torch.float64, device="cuda") for _ in range(2)]
            ptrs = [_dptr(t) for t in out]
        else:
            out = [np.empty(self.shape()) for _ in range(2)]
            ptrs = [_hptr(a) for a in out]
        _lcheck(load().fdcgks_line_get_state(self._h, *ptrs, int(device)), self._h)
        return tuple(out)

    def steps(self, dt, n):
        _lcheck(load().fdcgks_line_steps(self._h, ctypes.c_double(dt), int(n)), self._h)

    def run(self, t_end, cfl=0.4, max_steps=1 << 30):
        """Each line to t_end with its own CFL steps; returns (t [batch], steps [batch])."""
        t = np.zeros(self.batch)
        k = np.zeros(self.batch, dtype=np.int32)
        _lcheck(load().fdcgks_line_run(self._h, ctypes.c_double(t_end), ctypes.c_double(cfl), int(max_steps),
                                       t.ctypes.data, k.ctypes.data), self._h)
        return t, k

    def stage_operator(self, dt):
        import torch
        out = {k: torch.empty(self.shape(), dtype=torch.float64, device="cuda") for k in ("L", "Lt", "gb", "gt")}
        _lcheck(load().fdcgks_line_stage_operator(self._h, ctypes.c_double(dt),
                                                  *(_dptr(out[k]) for k in ("L", "Lt", "gb", "gt"))), self._h)
        return out

    def check(self):
        """(per-line status bits, their OR): bit 0 non-physical node, bit 1 no CFL time step."""
        flags = np.zeros(self.batch, dtype=np.int32)
        anyf = ctypes.c_int()
        _lcheck(load().fdcgks_line_check(self._h, flags.ctypes.data, ctypes.byref(anyf)), self._h)
        return flags, anyf.value


def _steps_function():
    import torch

    class StepsFunction(torch.autograd.Function):
        """Differentiable n-step FD-CGKS map (FP64 contexts): forward runs the
        library's steps, backward its adjoint (fdcgks_vjp_steps)."""

        @staticmethod
        def forward(ctx, Wp, Gp, Wd, Gd, solver, dt, nsteps, checkpoint_every):
            state0 = tuple(t.detach().contiguous() for t in (Wp, Gp, Wd, Gd))
            solver.set_state(*state0)
            solver.steps(dt, nsteps)
            out = solver.get_state()
            torch.cuda.current_stream().synchronize()
            ctx.solver, ctx.dt, ctx.nsteps, ctx.ck = solver, dt, nsteps, checkpoint_every
            ctx.save_for_backward(*state0)
            return out

        @staticmethod
        def backward(ctx, gWp, gGp, gWd, gGd):
            state0 = ctx.saved_tensors
            adj = []
            for g, s in zip((gWp, gGp, gWd, gGd), state0):
                adj.append(torch.zeros_like(s) if g is None else g.contiguous().to(torch.float64))
            grads = ctx.solver.vjp_steps(ctx.dt, ctx.nsteps, state0, adj, ctx.ck)
            return grads + (None, None, None, None)

    return StepsFunction


_STEPS_FN = None


def steps_autograd(solver, Wp, Gp, Wd, Gd, dt, nsteps, checkpoint_every=50):
    """(Wp, Gp, Wd, Gd) after nsteps steps, differentiable with torch.autograd
    (the backward pass runs the library's adjoint kernels)."""
    global _STEPS_FN
    if _STEPS_FN is None:
        _STEPS_FN = _steps_function()
    return _STEPS_FN.apply(Wp, Gp, Wd, Gd, solver, dt, nsteps, checkpoint_every)
