"""Python binding of libbae (include/bae.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors (device memory) or numpy arrays (host memory) into plain pointers,
calls the C entry point with the same name and turns error codes into
exceptions. There is no fallback: if libbae.so is missing or no GPU is
usable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbae.so")

OK, ERR_INVALID_ARG, ERR_GEOMETRY, ERR_OOM, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA = range(7)
LAYER_DOUBLE, LAYER_SINGLE, LAYER_DIRECT = 0, 1, 2
FP64, MIXED, FP32, DF64 = 0, 1, 2, 3
_LAYERS = {"double": LAYER_DOUBLE, "single": LAYER_SINGLE, "direct": LAYER_DIRECT}
_PREC = {"fp64": FP64, "mixed": MIXED, "fp32": FP32, "df64": DF64}


class BAEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[bae error {code}] {msg}")
        self.code = code


class NotConverged(BAEError):
    pass


class GeometryError(BAEError):
    pass


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("restart", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_refine", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("residual_precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("particular", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("applies_fp64", ctypes.c_int),
                ("applies_fp32", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


BOUNDARY_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("h", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("phi", ctypes.c_void_p), ("kappa2", ctypes.c_double), ("layer", ctypes.c_int),
                ("f", ctypes.c_void_p), ("boundary", BOUNDARY_FN), ("user", ctypes.c_void_p),
                ("u_out", ctypes.c_void_p), ("opts", Options)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_gm", ctypes.c_int64), ("stats", Stats),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


PENDING = 7
_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def lib():
    """Loads libbae.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_05507_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "bae_version": (_I, []),
            "bae_last_error": (ctypes.c_char_p, []),
            "bae_default_options": (None, [_P]),
            "bae_launch_count": (ctypes.c_longlong, []),
            "bae_set_conv_schedule": (_I, [_I]),
            "bae_inject_fault": (_I, [_I, ctypes.c_longlong]),
            "bae_profile_start": (_I, [_I]),
            "bae_profile_stop": (_I, [ctypes.c_char_p, _I, _P, _P, _I, _P]),
            "bae_ctx_create": (_I, [_I, _P, _P]),
            "bae_ctx_destroy": (None, [_P]),
            "bae_lgf_table": (_I, [_P, _I, _D, _P]),
            "bae_lgf_spectrum": (_I, [_P, _I, _D, _P]),
            "bae_problem_create": (_I, [_P, _I, _D, _P, _P, _D, _I, _P]),
            "bae_problem_destroy": (None, [_P]),
            "bae_problem_sizes": (_I, [_P, _P, _P, _P]),
            "bae_problem_unknowns": (_I, [_P, _P]),
            "bae_gamma_plus": (_I, [_P, _P]),
            "bae_interior_mask": (_I, [_P, _P]),
            "bae_problem_plane_range": (_I, [_P, _P, _P]),
            "bae_problem_conv_planes": (_I, [_P, _P, _P, _P]),
            "bae_boundary_points": (_I, [_P, _P]),
            "bae_classification": (_I, [_P, _P, _P, _P, _P]),
            "bae_potential_apply": (_I, [_P, _I, _P, _P]),
            "bae_potential_apply_noalloc": (_I, [_P, _I, _P, _P]),
            "bae_boundary_apply": (_I, [_P, _I, _P, _P]),
            "bae_particular": (_I, [_P, _I, _P, _P]),
            "bae_box_particular": (_I, [_P, _I, _P, _P]),
            "bae_solve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
            "bae_solve_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
            "bae_server_create": (_I, [_I, _I, ctypes.c_int64, _P]),
            "bae_server_submit": (_I, [_P, _P, _P]),
            "bae_server_poll": (_I, [_P, ctypes.c_int64, _I, _P]),
            "bae_server_density": (_I, [_P, ctypes.c_int64, _P, ctypes.c_int64]),
            "bae_server_release": (_I, [_P, ctypes.c_int64]),
            "bae_server_clock": (_D, [_P]),
            "bae_server_destroy": (None, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


EXPORTED = ["bae_version", "bae_last_error", "bae_default_options", "bae_launch_count", "bae_set_conv_schedule",
            "bae_inject_fault", "bae_profile_start",
            "bae_profile_stop", "bae_ctx_create", "bae_ctx_destroy",
            "bae_lgf_table", "bae_lgf_spectrum", "bae_problem_create", "bae_problem_destroy",
            "bae_problem_sizes", "bae_problem_unknowns", "bae_gamma_plus", "bae_interior_mask", "bae_problem_plane_range",
            "bae_problem_conv_planes", "bae_boundary_points", "bae_classification", "bae_potential_apply",
            "bae_potential_apply_noalloc",
            "bae_boundary_apply", "bae_particular", "bae_box_particular", "bae_solve", "bae_solve_batched", "bae_server_create",
            "bae_server_submit", "bae_server_poll", "bae_server_density", "bae_server_release", "bae_server_clock",
            "bae_server_destroy"]


def _check(rc: int, allow_not_converged=False):
    if rc == OK:
        return
    msg = lib().bae_last_error().decode(errors="replace")
    if rc == ERR_NOT_CONVERGED:
        if allow_not_converged:
            return
        raise NotConverged(rc, msg)
    if rc == ERR_GEOMETRY:
        raise GeometryError(rc, msg)
    raise BAEError(rc, msg)


def _ptr(a):
    """Device pointer of a contiguous torch tensor, or host pointer of a
    contiguous numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _torch():
    import torch
    return torch


def _new(shape, dtype, like):
    """Output buffer matching the memory kind of `like` (torch on its device,
    else numpy on the host)."""
    if isinstance(like, np.ndarray) or like is None:
        return np.empty(shape, dtype=dtype)
    torch = _torch()
    tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
    return torch.empty(shape, dtype=tdt, device=like.device)


def _as_f64(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    torch = _torch()
    return a.to(torch.float64).contiguous()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().bae_launch_count())


FAULT_NONE, FAULT_BARRIER, FAULT_ALLOC_CAP = 0, 1, 2


def inject_fault(kind: int, arg: int = 0):
    """bae_inject_fault: host-side fault injection for failure tests."""
    _check(lib().bae_inject_fault(int(kind), int(arg)))


SCHEDULES = {"auto": -1, "passes": 0, "plane": 1, "passes_alt": 2, "persist": 3}


def set_conv_schedule(schedule: str = "auto"):
    """Forces the FFT convolution schedule of every potential apply in this
    process: "passes" (five kernels), "passes_alt" (the same with the second
    launch geometry), "persist" (the five as persistent kernels), "plane" (k
    and j fused per x-plane) or "auto" (every runnable schedule timed once
    per precision, N and batch size)."""
    if schedule not in SCHEDULES:
        raise ValueError(f"schedule must be one of {sorted(SCHEDULES)}")
    _check(lib().bae_set_conv_schedule(SCHEDULES[schedule]))


def profile_start(max_launches: int = 200000):
    _check(lib().bae_profile_start(int(max_launches)))


def profile_stop(max_kernels: int = 128) -> dict:
    """{kernel name: (total device ms, launches)} since profile_start."""
    names = ctypes.create_string_buffer(16384)
    ms = np.zeros(max_kernels)
    cnt = np.zeros(max_kernels, dtype=np.int64)
    nk = ctypes.c_int()
    _check(lib().bae_profile_stop(names, len(names), ms.ctypes.data, cnt.ctypes.data, max_kernels,
                                  ctypes.byref(nk)))
    keys = names.value.decode().split("\n")[: nk.value]
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(keys)}


class Context:
    """bae_ctx: one CUDA device and stream, with the LGF spectrum cache."""

    def __init__(self, device: int = 0, stream=None):
        """stream: a torch.cuda.Stream (or None for a new one). All library
        work of this context runs on it; record timing events on ctx.stream."""
        self.device = device
        self._h = ctypes.c_void_p()
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        _check(lib().bae_ctx_create(device, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().bae_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lgf_table(self, N: int, s: float, out=None):
        ntri = N * (N + 1) * (N + 2) // 6
        out = np.empty(ntri) if out is None else out
        _check(lib().bae_lgf_table(self._h, N, float(s), _ptr(out)))
        return out

    def lgf_spectrum(self, N: int, s: float, out=None):
        out = np.empty((N + 1,) * 3) if out is None else out
        _check(lib().bae_lgf_spectrum(self._h, N, float(s), _ptr(out)))
        return out


class Problem:
    """bae_problem: classified grid, closure, source stencil and spectrum."""

    def __init__(self, ctx: Context, phi, h: float, origin, kappa2: float = 0.0, layer: str = "double"):
        self.ctx = ctx
        phi = _as_f64(phi)
        self.N = int(phi.shape[0])
        self.h = float(h)
        o = np.array(origin if np.ndim(origin) else [origin] * 3, dtype=np.float64)
        self.origin = o
        self.kappa2 = float(kappa2)
        self.layer = layer
        self._h = ctypes.c_void_p()
        _check(lib().bae_problem_create(ctx._h, self.N, self.h, o.ctypes.data, _ptr(phi), self.kappa2,
                                        _LAYERS[layer], ctypes.byref(self._h)))
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bae_problem_sizes(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        self.n_gm, self.n_gp, self.n_mp = a.value, b.value, c.value
        _check(lib().bae_problem_unknowns(self._h, ctypes.byref(a)))
        self.n_unknowns = a.value   # n_gm, or n_gm + n_gp for the direct formulation

    def close(self):
        if self._h:
            lib().bae_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plane_range(self):
        """(lo, hi): the x-planes that hold every source and read-back node."""
        lo, hi = ctypes.c_int(), ctypes.c_int()
        _check(lib().bae_problem_plane_range(self._h, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def conv_planes(self):
        """(axis, lo, hi): the axis (0 x, 1 y, 2 z) and plane range that the
        convolutions inside a solve transform."""
        ax, lo, hi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bae_problem_conv_planes(self._h, ctypes.byref(ax), ctypes.byref(lo), ctypes.byref(hi)))
        return ax.value, lo.value, hi.value

    def boundary_points(self, like=None):
        out = _new((self.n_gm, 3), np.float64, like)
        _check(lib().bae_boundary_points(self._h, _ptr(out)))
        return out

    def classification(self):
        N = self.N
        flags = np.empty((N, N, N), np.uint8)
        gm = np.empty(self.n_gm, np.int32)
        partner = np.empty(self.n_gm, np.int32)
        t = np.empty(self.n_gm, np.float64)
        _check(lib().bae_classification(self._h, _ptr(flags), _ptr(gm), _ptr(partner), _ptr(t)))
        return dict(flags=flags, gm=gm, partner=partner, t=t)

    def interior_mask(self):
        """M+ as a bool array (N, N, N)."""
        m = np.empty((self.N,) * 3, np.uint8)
        _check(lib().bae_interior_mask(self._h, _ptr(m)))
        return m.astype(bool)

    def gamma_plus(self):
        """Linear indices of gamma+ (lexicographic)."""
        gp = np.empty(self.n_gp, np.int32)
        _check(lib().bae_gamma_plus(self._h, _ptr(gp)))
        return gp

    def potential_apply(self, q, precision="fp64", out=None):
        q = _as_f64(q)
        out = _new((self.N,) * 3, np.float64, q) if out is None else out
        _check(lib().bae_potential_apply(self._h, _PREC[precision], _ptr(q), _ptr(out)))
        return out

    def potential_apply_noalloc(self, q, out, precision="fp64"):
        """bae_potential_apply_noalloc: q and out must be CUDA tensors; the
        call allocates no device memory (static 8 MiB scratch)."""
        _check(lib().bae_potential_apply_noalloc(self._h, _PREC[precision], _ptr(q), _ptr(out)))
        return out

    def boundary_apply(self, q, precision="fp64", out=None):
        q = _as_f64(q)
        out = _new((self.n_unknowns,), np.float64, q) if out is None else out
        _check(lib().bae_boundary_apply(self._h, _PREC[precision], _ptr(q), _ptr(out)))
        return out

    def box_particular(self, f, precision="fp64", out=None):
        """bae_box_particular: u_p on the finite auxiliary box of eq. [aux]."""
        f = _as_f64(f)
        out = _new((self.N,) * 3, np.float64, f) if out is None else out
        _check(lib().bae_box_particular(self._h, _PREC[precision], _ptr(f), _ptr(out)))
        return out

    def particular(self, f, precision="fp64", out=None):
        f = _as_f64(f)
        out = _new((self.N,) * 3, np.float64, f) if out is None else out
        _check(lib().bae_particular(self._h, _PREC[precision], _ptr(f), _ptr(out)))
        return out

    def _opts(self, tol, precision, max_iter, restart, max_refine, inner_tol, use_graphs=False,
              residual_precision=None, precond=None, particular=None):
        o = Options()
        lib().bae_default_options(ctypes.byref(o))
        if particular is not None:   # "lattice" (free-lattice G_h) or "box" (eq. [aux])
            o.particular = {"lattice": 0, "box": 1}[particular]
        o.use_graphs = 1 if use_graphs else 0
        if precond is not None:   # False/0: never, True/1: every refinement step, 2: after the first
            o.precond = int(precond)
        if residual_precision is not None:
            o.residual_precision = _PREC[residual_precision]
        o.tol = tol
        o.precision = _PREC[precision]
        if max_iter is not None:
            o.max_iter = max_iter
        if restart is not None:
            o.restart = restart
        if max_refine is not None:
            o.max_refine = max_refine
        if inner_tol is not None:
            o.inner_tol = inner_tol
        return o

    def solve(self, f, g, tol=1e-10, precision="fp64", max_iter=None, restart=None, max_refine=None,
              inner_tol=None, density=None, u=None, allow_not_converged=False, use_graphs=False,
              residual_precision=None, precond=None, particular=None):
        """Returns (density, u, stats dict). f (N^3) and g (n_gm) may be
        torch CUDA tensors or numpy arrays; outputs follow f's kind."""
        f = _as_f64(f)
        g = _as_f64(g)
        density = _new((self.n_unknowns,), np.float64, f) if density is None else density
        u = _new((self.N,) * 3, np.float64, f) if u is None else u
        st = Stats()
        o = self._opts(tol, precision, max_iter, restart, max_refine, inner_tol, use_graphs, residual_precision,
                       precond, particular)
        rc = lib().bae_solve(self._h, _ptr(f), _ptr(g), ctypes.byref(o), _ptr(density), _ptr(u), ctypes.byref(st))
        _check(rc, allow_not_converged)
        return density, u, st.as_dict()

    def solve_batched(self, f, g, tol=1e-10, precision="fp64", max_iter=None, restart=None, max_refine=None,
                      inner_tol=None, density=None, u=None, allow_not_converged=False, use_graphs=False,
                      residual_precision=None, precond=None):
        """f [nrhs, N, N, N], g [nrhs, n_gm]; returns (density, u, [stats])."""
        f = _as_f64(f)
        g = _as_f64(g)
        nrhs = int(f.shape[0])
        density = _new((nrhs, self.n_unknowns), np.float64, f) if density is None else density
        u = _new((nrhs,) + (self.N,) * 3, np.float64, f) if u is None else u
        st = (Stats * nrhs)()
        o = self._opts(tol, precision, max_iter, restart, max_refine, inner_tol, use_graphs, residual_precision,
                       precond)
        rc = lib().bae_solve_batched(self._h, nrhs, _ptr(f), _ptr(g), ctypes.byref(o), _ptr(density), _ptr(u),
                                     st)
        _check(rc, allow_not_converged)
        return density, u, [s.as_dict() for s in st]


class Server:
    """bae_server: continuous admission of solves into concurrent slots.
    Arrays passed to submit() are kept alive here until release()."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget_bytes: int = 64 << 30):
        self._h = ctypes.c_void_p()
        _check(lib().bae_server_create(device, slots, int(hbm_budget_bytes), ctypes.byref(self._h)))
        self._live = {}

    def close(self):
        if self._h:
            lib().bae_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clock(self) -> float:
        return float(lib().bae_server_clock(self._h))

    def submit(self, phi, h, origin, f, g_fn, kappa2=0.0, layer="double", u_out=None, tol=1e-10,
               precision="mixed", **opts) -> int:
        """g_fn(xyz (n,3) numpy) -> g (n,) numpy, called on a server thread."""
        phi = _as_f64(phi)
        f = _as_f64(f)
        N = int(phi.shape[0])
        if u_out is None:
            u_out = _new((N,) * 3, np.float64, f)

        def cb(xyz_p, n, g_p, _user):
            try:
                xyz = np.ctypeslib.as_array(xyz_p, shape=(int(n) * 3,)).reshape(-1, 3)
                gv = np.asarray(g_fn(xyz), dtype=np.float64).reshape(-1)
                np.ctypeslib.as_array(g_p, shape=(int(n),))[:] = gv
            except Exception as e:  # keep the server thread alive; g stays 0
                print("boundary callback failed:", e)

        fn = BOUNDARY_FN(cb)
        rq = Request()
        rq.N = N
        rq.h = float(h)
        o = np.array(origin if np.ndim(origin) else [origin] * 3, dtype=np.float64)
        for i in range(3):
            rq.origin[i] = o[i]
        rq.phi = _ptr(phi)
        rq.kappa2 = float(kappa2)
        rq.layer = _LAYERS[layer]
        rq.f = _ptr(f)
        rq.boundary = fn
        rq.user = None
        rq.u_out = _ptr(u_out)
        lib().bae_default_options(ctypes.byref(rq.opts))
        rq.opts.tol = tol
        rq.opts.precision = _PREC[precision]
        for k, v in opts.items():
            setattr(rq.opts, k, _PREC[v] if k == "residual_precision" else v)
        ticket = ctypes.c_int64()
        _check(lib().bae_server_submit(self._h, ctypes.byref(rq), ctypes.byref(ticket)))
        self._live[ticket.value] = (phi, f, u_out, fn, rq)
        return ticket.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Result dict when done (timeout_ms < 0 waits), else None."""
        res = Result()
        rc = lib().bae_server_poll(self._h, ticket, timeout_ms, ctypes.byref(res))
        if rc == PENDING:
            return None
        _check(rc)
        d = {k: getattr(res, k) for k, _ in Result._fields_ if k != "stats"}
        d["stats"] = res.stats.as_dict()
        d["u"] = self._live[ticket][2]
        return d

    def density(self, ticket: int):
        n = self.poll(ticket, 0)["n_gm"]
        out = np.empty(n)
        _check(lib().bae_server_density(self._h, ticket, out.ctypes.data, n))
        return out

    def release(self, ticket: int):
        _check(lib().bae_server_release(self._h, ticket))
        self._live.pop(ticket, None)
