"""Thin ctypes binding of libjko (include/jko.h), same names as the C ABI.

Argument marshalling only: every step of the JKO path runs in the CUDA
library.  PyTorch provides device memory and streams; energy fields are
passed as host float64 arrays and copied by ``jko_create``.  If libjko.so has
not been built the binding raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import enum
import math
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libjko.so")


class Precision(enum.IntEnum):
    FP64 = 0
    FP32 = 1
    TF32 = 2
    BF16 = 3
    BF16X3 = 4


class Status(enum.IntEnum):
    OK = 0
    INVALID_ARG = 1
    CUDA = 2
    OOM = 3
    NUMERIC = 4
    NOT_CONVERGED = 5
    TIMEOUT = 6
    UNSUPPORTED = 7


class JKOError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{Status(status).name}: {message}")
        self.status = Status(status)
        self.message = message


class jko_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("heat_L", ctypes.c_int),
                ("fft", ctypes.c_int)]


class jko_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("precision", ctypes.c_int), ("renormalize", ctypes.c_int),
                ("absorb", ctypes.c_int),
                ("loop", ctypes.c_int),
                ("tile", ctypes.c_int),
                ("stall", ctypes.c_int),
                ("finish", ctypes.c_int)]


class jko_energy(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("kappa", ctypes.c_double),
                ("kappa_field", ctypes.c_void_p), ("m", ctypes.c_double),
                ("alpha", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("m_field", ctypes.c_void_p), ("binary", ctypes.c_int),
                ("target", ctypes.c_void_p), ("species", ctypes.c_int),
                ("w2", ctypes.c_void_p), ("pair_alpha", ctypes.c_double)]


class jko_step_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("residual_l1", ctypes.c_double), ("mass", ctypes.c_double),
                ("max_p_over_kappa", ctypes.c_double), ("ms", ctypes.c_float),
                ("kernels", ctypes.c_int), ("iters_finish", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = {
    "jko_create": (ctypes.c_int, [ctypes.POINTER(jko_grid), ctypes.POINTER(jko_params),
                                  ctypes.POINTER(jko_energy), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "jko_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.POINTER(jko_step_info)]),
    "jko_flow": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(jko_step_info)]),
    "jko_flow_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(jko_step_info)]),
    "jko_profile_passes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_double)]),
    "jko_profile_loop": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_double)]),
    "jko_handle_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "jko_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "jko_step_noalloc": (ctypes.c_int, [ctypes.POINTER(jko_grid), ctypes.POINTER(jko_params),
                                        ctypes.POINTER(jko_energy), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(jko_step_info)]),
    "jko_set_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "jko_set_potential_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "jko_flow_record": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.POINTER(jko_step_info)]),
    "jko_flow_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "jko_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(jko_grid),
                                        ctypes.POINTER(jko_params), ctypes.POINTER(jko_energy),
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "jko_batch_flow": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(jko_step_info)]),
    "jko_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(jko_step_info)]),
    "jko_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "jko_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "jko_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "jko_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "jko_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "jko_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "jko_build_info": (ctypes.c_char_p, []),
    "jko_heat_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libjko.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, handle=None) -> int:
    if status in (Status.OK, Status.NOT_CONVERGED, Status.NUMERIC):
        return status
    msg = lib().jko_last_error(handle).decode(errors="replace")
    raise JKOError(status, msg)


def _host_f64(x, N) -> Optional[np.ndarray]:
    if x is None:
        return None
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), (N,)))
    return a


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Handle:
    """Owns a jko_handle*; keeps the parameters used to create it."""

    def __init__(self, ptr: ctypes.c_void_p, nx: int, ny: int, precision: Precision,
                 species: int = 1):
        self.ptr = ptr
        self.nx, self.ny = nx, ny
        self.cells = nx * ny                             # elements of a field (w, kappa)
        self.N = self.cells * (2 if species == 2 else 1)  # elements of a state image
        self.precision = Precision(precision)

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == Precision.FP64 else torch.float32

    @property
    def np_dtype(self):
        return np.float64 if self.precision == Precision.FP64 else np.float32

    def __del__(self):
        try:
            if self.ptr:
                jko_destroy(self)
        except Exception:
            pass


def jko_create(nx: int, ny: int, gamma: float, tau: float, *, lx: float = 1.0, ly: float = 1.0,
               tol: float = 1e-6, max_iter: int = 200, check_every: int = 0,
               precision: int = Precision.FP32, renormalize: bool = True,
               w=None, kappa: float = math.inf, kappa_field=None, m: float = 0.0,
               alpha=None, mask=None, stream=None, absorb: int = 0, loop: int = 0,
               tile: int = 0, m_field=None, binary: bool = False, target=None,
               species: int = 1, w2=None, heat_L: int = 0,
               pair_alpha: float = 0.0, stall: int = 0, finish: int = 0,
               fft: int = 0) -> Handle:
    """jko_create: grid, step parameters and energy (host arrays, copied);
    ``m_field``: per-cell exponents of the paper's generalised entropies;
    ``binary``: the non-convex congestion iota_{{0,kappa}}; ``target``: the
    density r of the Wasserstein attraction (Sec. 5.2); ``species = 2`` with
    ``w2``: two densities coupled through the congestion of their sum (Sec. 5.3),
    or with ``pair_alpha > 0`` through the pairwise attraction pair_alpha
    W(p_1, p_2), whose state images hold [p_1, p_2]; ``heat_L > 0``: the heat-kernel Gibbs
    kernel (Id - (gamma/L) Delta)^{-L} of the domain outside ``mask`` (Sec. 4.1);
    ``stall > 0``: a step also stops when its residual sets no new minimum for
    that many pairs; ``finish = 1`` (tensor-core precisions): such a step goes
    on from its scalings on the FP32 CUDA-core form until tol; ``fft = 1``:
    the Gaussian applied by FFT convolution along each axis."""
    N = nx * ny
    g = jko_grid(nx, ny, lx, ly, int(heat_L), int(fft))
    p = jko_params(gamma, tau, tol, max_iter, check_every, int(precision), int(bool(renormalize)),
                   int(absorb), int(loop), int(tile), int(stall), int(finish))
    keep = [_host_f64(w, N), _host_f64(kappa_field, N), _host_f64(alpha, N),
            _host_f64(m_field, N), _host_f64(target, N), _host_f64(w2, N)]
    mk = None if mask is None else np.ascontiguousarray(np.asarray(mask, np.uint8).reshape(N))
    e = jko_energy(keep[0].ctypes.data if keep[0] is not None else None, float(kappa),
                   keep[1].ctypes.data if keep[1] is not None else None, float(m),
                   keep[2].ctypes.data if keep[2] is not None else None,
                   mk.ctypes.data if mk is not None else None,
                   keep[3].ctypes.data if keep[3] is not None else None, int(bool(binary)),
                   keep[4].ctypes.data if keep[4] is not None else None, int(species),
                   keep[5].ctypes.data if keep[5] is not None else None, float(pair_alpha))
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(lib().jko_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(e), st,
                            ctypes.byref(out)))
    return Handle(out, nx, ny, precision, species)


def _dev_image(h: Handle, t, name, n=None):
    import torch
    n = h.N if n is None else n
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != h.dtype or not t.is_contiguous() or t.numel() < n:
        raise TypeError(f"{name} must be a contiguous {h.dtype} tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def jko_step(h: Handle, q, p_out=None):
    """One JKO step on device tensors; returns (p_out, info dict)."""
    import torch
    if p_out is None:
        p_out = torch.empty(h.N, dtype=h.dtype, device=q.device)
    info = jko_step_info()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_step(h.ptr, _dev_image(h, q, "q"), _dev_image(h, p_out, "p_out"),
                      ctypes.byref(info)), h.ptr)
    return p_out, info.as_dict()


def jko_flow(h: Handle, p0, n_steps: int, traj=None, p_final=None, want_traj: bool = True):
    """n_steps of the flow on device tensors; returns (p_final, traj, infos)."""
    import torch
    if traj is None and want_traj and n_steps > 0:
        traj = torch.empty((n_steps, h.N), dtype=h.dtype, device=p0.device)
    if p_final is None:
        p_final = torch.empty(h.N, dtype=h.dtype, device=p0.device)
    infos = (jko_step_info * max(n_steps, 1))()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    tptr = _dev_image(h, traj.reshape(-1), "traj") if traj is not None else None
    _check(L.jko_flow(h.ptr, _dev_image(h, p0, "p0"), n_steps, tptr,
                      _dev_image(h, p_final, "p_final"), infos), h.ptr)
    return p_final, traj, [infos[i].as_dict() for i in range(n_steps)]


def jko_flow_host(h: Handle, p0_host, n_steps: int, traj_host=None, p_final_host=None):
    """The flow on host buffers (numpy arrays or pinned CPU tensors)."""
    def ptr(x):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            if x.dtype != h.np_dtype or not x.flags.c_contiguous:
                raise TypeError(f"host buffer must be a contiguous {h.np_dtype} array")
            return ctypes.c_void_p(x.ctypes.data)
        return ctypes.c_void_p(x.data_ptr())
    infos = (jko_step_info * max(n_steps, 1))()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_flow_host(h.ptr, ptr(p0_host), n_steps, ptr(traj_host), ptr(p_final_host),
                           infos), h.ptr)
    return [infos[i].as_dict() for i in range(n_steps)]


def jko_profile_passes(h: Handle, reps: int = 20):
    """Mean ms per launch and algorithmic flops of the four passes of a pair."""
    ms = (ctypes.c_float * 4)()
    fl = (ctypes.c_double * 4)()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_profile_passes(h.ptr, reps, ms, fl), h.ptr)
    return list(ms), list(fl)


def jko_profile_loop(h: Handle, pairs: int = 16, reps: int = 10):
    """Mean ms per launch and executed flops of the persistent pair-loop kernel
    running `pairs` pairs."""
    ms = (ctypes.c_float * 1)()
    fl = (ctypes.c_double * 1)()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_profile_loop(h.ptr, pairs, reps, ms, fl), h.ptr)
    return ms[0], fl[0]


def jko_handle_info(h: Handle) -> dict:
    """Which kernels a handle runs: persistent loop kernel, resident factor
    band, graph replay, pairs per launch or chunk."""
    out = (ctypes.c_int * 4)()
    _check(lib().jko_handle_info(h.ptr, out), h.ptr)
    return {"loop": bool(out[0]), "resident": bool(out[1]), "graph": bool(out[2]),
            "pairs_per_launch": int(out[3])}


def jko_batch_info(b) -> dict:
    """The batch autotuner's choice: 'tuned' (-1 none, 0 each flow's own, 1
    per-pass 64, 2 per-pass 128, 3 loop kernel, 4 grouped launches), flows on
    a loop-kernel launch of their own, whether the per-pass fallback was
    taken, flows in grouped launches and the number of grouped launches."""
    out = (ctypes.c_int * 5)()
    _check(lib().jko_batch_info(b.ptr, out), None)
    return {"tuned": int(out[0]), "loop_flows": int(out[1]), "per_pass_fallback": bool(out[2]),
            "grouped_flows": int(out[3]), "grouped_launches": int(out[4])}


def jko_step_noalloc(pb, q, p_out, tol: Optional[float] = None,
                     max_iter: Optional[int] = None, renormalize: bool = True):
    """jko_step_noalloc for an ``inputs.Problem``: one FP32 step whose working
    buffers live in the library's fixed device array (nothing is allocated by
    the library; q and p_out are caller-owned float32 CUDA tensors).  Returns
    (status, info dict); raises on errors other than NOT_CONVERGED/NUMERIC."""
    N = pb.nx * pb.ny
    for t, name in ((q, "q"), (p_out, "p_out")):
        if not t.is_cuda or str(t.dtype) != "torch.float32" or not t.is_contiguous() \
                or t.numel() < N:
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor of {N} elements")
    g = jko_grid(pb.nx, pb.ny, pb.lx, pb.ly, int(getattr(pb, "heat_L", 0)))
    p = jko_params(pb.gamma, pb.tau, pb.tol if tol is None else tol,
                   pb.max_iter if max_iter is None else max_iter, 0, int(Precision.FP32),
                   int(bool(renormalize)), 0)
    keep = [_host_f64(pb.w, N), None, _host_f64(pb.alpha, N),
            _host_f64(getattr(pb, "m_field", None), N), _host_f64(getattr(pb, "target", None), N)]
    mk = None if pb.mask is None else np.ascontiguousarray(np.asarray(pb.mask, np.uint8).reshape(N))
    e = jko_energy(keep[0].ctypes.data if keep[0] is not None else None, float(pb.kappa), None,
                   float(pb.m), keep[2].ctypes.data if keep[2] is not None else None,
                   mk.ctypes.data if mk is not None else None,
                   keep[3].ctypes.data if keep[3] is not None else None,
                   int(bool(getattr(pb, "binary", False))),
                   keep[4].ctypes.data if keep[4] is not None else None,
                   int(getattr(pb, "species", 1)))
    info = jko_step_info()
    st = lib().jko_step_noalloc(ctypes.byref(g), ctypes.byref(p), ctypes.byref(e),
                                ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p_out.data_ptr()),
                                _current_stream(), ctypes.byref(info))
    if st not in (Status.OK, Status.NOT_CONVERGED, Status.NUMERIC):
        raise JKOError(st, "jko_step_noalloc failed (see the status code)")
    return Status(st), info.as_dict()


def jko_destroy(h: Handle) -> None:
    if h.ptr:
        lib().jko_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


def jko_last_error(h: Optional[Handle] = None) -> str:
    return lib().jko_last_error(h.ptr if h else None).decode(errors="replace")


def jko_build_info() -> str:
    return lib().jko_build_info().decode()


def jko_heat_plan(nx: int, ny: int, gamma: float, L: int = 10, lx: float = 1.0,
                  ly: float = 1.0, precision: int = Precision.FP64) -> dict:
    """jko_heat_plan (host only): the degree, Chebyshev coefficients and
    spectrum interval of the heat kernel's expansion."""
    deg = ctypes.c_int()
    iv = (ctypes.c_double * 2)()
    _check(lib().jko_heat_plan(nx, ny, lx, ly, gamma, L, int(precision), ctypes.byref(deg),
                               None, 0, iv))
    coef = (ctypes.c_double * (deg.value + 1))()
    _check(lib().jko_heat_plan(nx, ny, lx, ly, gamma, L, int(precision), ctypes.byref(deg),
                               coef, deg.value + 1, iv))
    return {"degree": deg.value, "coef": np.array(coef[:]), "interval": (iv[0], iv[1])}


def create_from_problem(pb, precision: int = Precision.FP32, tol: Optional[float] = None,
                        max_iter: Optional[int] = None, check_every: int = 0,
                        renormalize: bool = True, stream=None, absorb: int = 0,
                        loop: int = 0, tile: int = 0, stall: int = 0, finish: int = 0,
                        fft: int = 0) -> Handle:
    """jko_create from an ``inputs.Problem``."""
    return jko_create(pb.nx, pb.ny, pb.gamma, pb.tau, lx=pb.lx, ly=pb.ly,
                      tol=pb.tol if tol is None else tol,
                      max_iter=pb.max_iter if max_iter is None else max_iter,
                      check_every=check_every, precision=precision, renormalize=renormalize,
                      w=pb.w, kappa=pb.kappa, m=pb.m, alpha=pb.alpha, mask=pb.mask,
                      stream=stream, absorb=absorb, loop=loop, tile=tile,
                      m_field=getattr(pb, "m_field", None),
                      binary=bool(getattr(pb, "binary", False)),
                      target=getattr(pb, "target", None),
                      species=int(getattr(pb, "species", 1)), w2=getattr(pb, "w2", None),
                      heat_L=int(getattr(pb, "heat_L", 0)),
                      pair_alpha=float(getattr(pb, "pair_alpha", 0.0)), stall=stall,
                      finish=finish, fft=fft)


class Batch:
    """Owns a jko_batch*: independent flows advanced together."""

    def __init__(self, ptr, shapes, precisions):
        self.ptr = ptr
        self.shapes = shapes              # (nx, ny) per flow
        self.precisions = precisions

    @property
    def n(self):
        return len(self.shapes)

    def __del__(self):
        try:
            if self.ptr:
                jko_batch_destroy(self)
        except Exception:
            pass


def _energy_struct(pb, keep):
    N = pb.nx * pb.ny
    w, al = _host_f64(pb.w, N), _host_f64(pb.alpha, N)
    mk = None if pb.mask is None else np.ascontiguousarray(np.asarray(pb.mask, np.uint8).reshape(N))
    mf = _host_f64(getattr(pb, "m_field", None), N)
    tg = _host_f64(getattr(pb, "target", None), N)
    w2 = _host_f64(getattr(pb, "w2", None), N)
    keep += [w, al, mk, mf, tg, w2]
    return jko_energy(w.ctypes.data if w is not None else None, float(pb.kappa), None, float(pb.m),
                      al.ctypes.data if al is not None else None,
                      mk.ctypes.data if mk is not None else None,
                      mf.ctypes.data if mf is not None else None,
                      int(bool(getattr(pb, "binary", False))),
                      tg.ctypes.data if tg is not None else None,
                      int(getattr(pb, "species", 1)),
                      w2.ctypes.data if w2 is not None else None,
                      float(getattr(pb, "pair_alpha", 0.0)))


def jko_batch_create(problems, precision=Precision.FP32, tol=None, max_iter=None,
                     check_every: int = 0, renormalize: bool = True, stream=None,
                     loop: int = 0, tile: int = 0, stall: int = 0) -> Batch:
    """jko_batch_create for a list of ``inputs.Problem``; ``precision`` and
    ``loop`` may be one value or one per flow (loop = 3: grouped launch)."""
    n = len(problems)
    precs = list(precision) if isinstance(precision, (list, tuple)) else [precision] * n
    loops = list(loop) if isinstance(loop, (list, tuple)) else [loop] * n
    G = (jko_grid * n)()
    P = (jko_params * n)()
    E = (jko_energy * n)()
    keep = []
    for f, pb in enumerate(problems):
        G[f] = jko_grid(pb.nx, pb.ny, pb.lx, pb.ly, int(getattr(pb, "heat_L", 0)))
        P[f] = jko_params(pb.gamma, pb.tau, pb.tol if tol is None else tol,
                          pb.max_iter if max_iter is None else max_iter, check_every,
                          int(precs[f]), int(bool(renormalize)), 0, int(loops[f]), int(tile),
                          int(stall), 0)
        E[f] = _energy_struct(pb, keep)
    out = ctypes.c_void_p()
    st = _current_stream() if stream is None else ctypes.c_void_p(stream)
    status = lib().jko_batch_create(n, G, P, E, st, ctypes.byref(out))
    if status != Status.OK:
        raise JKOError(status, lib().jko_batch_last_error(None).decode(errors="replace"))
    return Batch(out, [(pb.nx, pb.ny) for pb in problems], [Precision(p) for p in precs])


def jko_batch_step(b: Batch, qs, p_outs=None):
    """One step of every flow from the device tensors qs into p_outs (new
    tensors when None); returns (p_outs, infos[f])."""
    import torch
    n = b.n
    outs = [torch.empty_like(t) for t in qs] if p_outs is None else list(p_outs)
    Q = (ctypes.c_void_p * n)(*[ctypes.c_void_p(t.data_ptr()) for t in qs])
    PO = (ctypes.c_void_p * n)(*[ctypes.c_void_p(t.data_ptr()) for t in outs])
    infos = (jko_step_info * n)()
    status = lib().jko_batch_step(b.ptr, Q, PO, infos)
    if status not in (Status.OK, Status.NOT_CONVERGED, Status.NUMERIC):
        raise JKOError(status, lib().jko_batch_last_error(b.ptr).decode(errors="replace"))
    return outs, [infos[f].as_dict() for f in range(n)]


def jko_batch_flow(b: Batch, p0s, n_steps: int, want_final: bool = True):
    """n_steps of every flow from the device tensors p0s; returns
    (final images, infos[t][f])."""
    import torch
    n = b.n
    P0 = (ctypes.c_void_p * n)(*[ctypes.c_void_p(t.data_ptr()) for t in p0s])
    finals = [torch.empty_like(t) for t in p0s] if want_final else None
    PF = (ctypes.c_void_p * n)(*[ctypes.c_void_p(t.data_ptr()) for t in finals]) if finals else None
    infos = (jko_step_info * max(1, n * n_steps))()
    status = lib().jko_batch_flow(b.ptr, P0, n_steps, PF, infos)
    if status not in (Status.OK, Status.NOT_CONVERGED, Status.NUMERIC):
        raise JKOError(status, lib().jko_batch_last_error(b.ptr).decode(errors="replace"))
    table = [[infos[t * n + f].as_dict() for f in range(n)] for t in range(n_steps)]
    return finals, table


def jko_batch_destroy(b: Batch) -> None:
    if b.ptr:
        lib().jko_batch_destroy(b.ptr)
        b.ptr = ctypes.c_void_p()


# ---- differentiation ---------------------------------------------------------------

def jko_set_potential(h: Handle, w) -> None:
    """Replaces the potential w (host float64 copy of any array-like)."""
    wh = _host_f64(np.asarray(w, np.float64).reshape(-1), h.cells)
    _check(lib().jko_set_potential(h.ptr, ctypes.c_void_p(wh.ctypes.data)), h.ptr)


def jko_set_potential_device(h: Handle, w) -> None:
    """Replaces the potential w from a device tensor (cast to the handle's
    element type), stream-ordered on the current stream."""
    wd = w.detach().to(h.dtype).contiguous()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_set_potential_device(h.ptr, _dev_image(h, wd, "w", h.cells)), h.ptr)
    return wd


def jko_flow_record(h: Handle, p0, n_steps: int):
    """jko_flow that records the tape for jko_flow_backward; returns (p_n, infos)."""
    import torch
    p_final = torch.empty(h.N, dtype=h.dtype, device=p0.device)
    infos = (jko_step_info * n_steps)()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_flow_record(h.ptr, _dev_image(h, p0, "p0"), n_steps,
                             _dev_image(h, p_final, "p_final"), infos), h.ptr)
    return p_final, [infos[i].as_dict() for i in range(n_steps)]


def jko_flow_backward(h: Handle, grad_final, want_p0: bool = True, want_w: bool = True):
    """dL/dp_0 and dL/dw of the last recorded flow, given dL/dp_n."""
    import torch
    gp = torch.empty(h.N, dtype=h.dtype, device=grad_final.device) if want_p0 else None
    gw = torch.empty(h.cells, dtype=h.dtype, device=grad_final.device) if want_w else None
    n = 4096
    iters = (ctypes.c_int * n)()
    L = lib()
    _check(L.jko_set_stream(h.ptr, _current_stream()), h.ptr)
    _check(L.jko_flow_backward(h.ptr, _dev_image(h, grad_final.contiguous(), "grad"),
                               _dev_image(h, gp, "grad_p0") if gp is not None else None,
                               _dev_image(h, gw, "grad_w", h.cells) if gw is not None else None,
                               iters), h.ptr)
    return gp, gw, list(iters)


def _autograd_function():
    import torch

    class JKOFlow(torch.autograd.Function):
        """p_n = flow(p_0, w) on a CUDA-core handle; backward through the
        library's implicit adjoint.  One recorded flow per handle at a time."""

        @staticmethod
        def forward(ctx, p0, w, handle, n_steps):
            if w.is_cuda:
                wd = jko_set_potential_device(handle, w)
            else:
                jko_set_potential(handle, w.detach().double().cpu().numpy())
            pT, _ = jko_flow_record(handle, p0.detach().to(handle.dtype).contiguous(), n_steps)
            if w.is_cuda:
                del wd      # flow_record synchronised: the potential kernel has run
            ctx.handle = handle
            ctx.w_meta = (w.dtype, w.device)
            ctx.p0_meta = (p0.dtype, p0.device)
            return pT

        @staticmethod
        def backward(ctx, grad):
            gp, gw, _ = jko_flow_backward(ctx.handle, grad.to(ctx.handle.dtype))
            return (gp.to(dtype=ctx.p0_meta[0], device=ctx.p0_meta[1]),
                    gw.to(dtype=ctx.w_meta[0], device=ctx.w_meta[1]), None, None)

    return JKOFlow


_JKOFlow = None


def jko_flow_autograd(p0, w, handle: Handle, n_steps: int):
    """Differentiable flow: returns p_n with gradients to p0 and w."""
    global _JKOFlow
    if _JKOFlow is None:
        _JKOFlow = _autograd_function()
    return _JKOFlow.apply(p0, w, handle, n_steps)
