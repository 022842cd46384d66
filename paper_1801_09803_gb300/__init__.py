"""Python binding of libxc (GB300 line-list -> cross-section engine).

This module only marshals arguments to the C ABI declared in ``include/xc.h``:
numpy arrays are passed as host pointers, CUDA torch tensors as device
pointers on torch's current stream.  Every step of the computation runs in the
library's CUDA kernels; if the library is missing this module raises instead
of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from . import build as _build

__all__ = [
    "XcError", "Engine", "partition_function", "lib", "LIB_PATH", "make_condition", "make_grid", "make_opts",
    "PROFILES", "PRECISIONS", "QUANTITIES", "THRESHOLDS", "make_broadener", "XC_MEM_HOST", "XC_MEM_DEVICE", "EXPORTED_SYMBOLS",
]

LIB_PATH = _build.LIB
XC_MEM_HOST, XC_MEM_DEVICE = 0, 1
PROFILES = {"doppler": 0, "lorentz": 1, "voigt_w4": 2, "voigt_gh_binned": 3, "voigt_gh_sampled": 4,
            "doppler_binned": 5, "lorentz_binned": 6, "voigt_vv": 7}
PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS = {0: "XC_OK", 1: "XC_EINVAL", 2: "XC_ENOMEM", 3: "XC_ECUDA", 4: "XC_ETIMEOUT", 5: "XC_EUNSUPPORTED"}
EXPORTED_SYMBOLS = [
    "xc_version", "xc_last_error", "xc_create", "xc_destroy", "xc_load_lines", "xc_num_lines", "xc_get_lines",
    "xc_get_permutation", "xc_set_states", "xc_partition_function", "xc_line_params", "xc_count_evals",
    "xc_cross_section", "xc_cross_section_batched", "xc_cross_section_vjp", "xc_set_timing", "xc_last_timings",
    "xc_get_tuning", "xc_last_launch_count", "xc_cross_section_batched_static", "xc_set_tile_shape",
    "xc_last_sweep_kernels", "xc_set_broadening", "xc_count_far_evals", "xc_cross_section_vjp_broadening",
]


class XcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class XcLines(C.Structure):
    _fields_ = [("nu", C.c_void_p), ("elower", C.c_void_p), ("A", C.c_void_p), ("gamma_ref", C.c_void_p),
                ("n_T", C.c_void_p), ("g_up", C.c_void_p), ("j_lo", C.c_void_p), ("mem", C.c_int)]


class XcCondition(C.Structure):
    _fields_ = [("T", C.c_double), ("P", C.c_double), ("Q", C.c_double), ("dQdT", C.c_double),
                ("mass_da", C.c_double), ("T_ref", C.c_double), ("P_ref", C.c_double),
                ("gamma_scale", C.c_double), ("n_shift", C.c_double), ("abundance", C.c_double)]


class XcGrid(C.Structure):
    _fields_ = [("nu_A", C.c_double), ("step", C.c_double), ("n", C.c_int64)]


class XcOpts(C.Structure):
    _fields_ = [("profile", C.c_int), ("precision", C.c_int), ("cutoff", C.c_double),
                ("width_mult", C.c_double), ("n_gh", C.c_int), ("flags", C.c_int),
                ("quantity", C.c_int), ("threshold", C.c_int), ("I_cut", C.c_double),
                ("nu_crit", C.c_double), ("I_crit", C.c_double), ("vv_split", C.c_double), ("vv_flags", C.c_int)]


QUANTITIES = {"absorption": 0, "emission": 1}
BROAD_TYPES = {"constant": 0, "a0": 1, "a1": 2}


class XcBroadener(C.Structure):
    _fields_ = [("type", C.c_int), ("fraction", C.c_double), ("gamma0", C.c_double), ("n", C.c_double),
                ("n_entries", C.c_int64), ("j_lo", C.c_void_p), ("j_up", C.c_void_p), ("gamma0_j", C.c_void_p),
                ("n_j", C.c_void_p)]


def make_broadener(kind: str, fraction: float, gamma0: float, n: float, table=None) -> XcBroadener:
    """One .broad broadener: kind "constant", "a0" (table {J'': (gamma0, n)}) or "a1" (table
    {(J'', J'): (gamma0, n)}); gamma0 / n are the defaults for lines the table does not list."""
    t = BROAD_TYPES[kind]
    rows = sorted((table or {}).items())
    jl = np.array([k if t == 1 else k[0] for k, _ in rows], np.int32)
    ju = np.array([k[1] for k, _ in rows] if t == 2 else [], np.int32)
    g0 = np.array([v[0] for _, v in rows], np.float64)
    nn = np.array([v[1] for _, v in rows], np.float64)
    b = XcBroadener(t, float(fraction), float(gamma0), float(n), len(rows), jl.ctypes.data,
                    ju.ctypes.data if t == 2 else None, g0.ctypes.data, nn.ctypes.data)
    b._keep = (jl, ju, g0, nn)   # the arrays the pointers refer to
    return b
THRESHOLDS = {"constant": 1, "hitran": 2}


_lib = None


def lib(build_if_missing: bool = False):
    """Load libxc.so.  Raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            _build.build()
        else:
            raise XcError(5, f"{LIB_PATH} is missing: run paper_1801_09803_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    vp, st, i, d = C.c_void_p, C.c_size_t, C.c_int, C.c_double
    sigs = {
        "xc_version": ([], C.c_char_p), "xc_last_error": ([], C.c_char_p),
        "xc_create": ([C.POINTER(vp), i], i), "xc_destroy": ([vp], i),
        "xc_load_lines": ([vp, C.POINTER(XcLines), st, C.c_uint, vp], i),
        "xc_num_lines": ([vp, C.POINTER(st)], i),
        "xc_get_lines": ([vp] + [vp] * 7 + [i, vp], i),
        "xc_get_permutation": ([vp, vp, i, vp], i),
        "xc_set_states": ([vp, vp, vp, st, i, vp], i),
        "xc_partition_function": ([vp, vp, st, vp, st, vp, vp, i, vp], i),
        "xc_line_params": ([vp, C.POINTER(XcCondition), vp, vp, vp, i, vp], i),
        "xc_count_evals": ([vp, C.POINTER(XcCondition), st, C.POINTER(XcGrid), C.POINTER(XcOpts),
                            C.POINTER(C.c_int64), vp], i),
        "xc_cross_section": ([vp, C.POINTER(XcCondition), C.POINTER(XcGrid), C.POINTER(XcOpts), vp, i, vp], i),
        "xc_cross_section_batched": ([vp, C.POINTER(XcCondition), st, C.POINTER(XcGrid), C.POINTER(XcOpts), vp,
                                      i, vp], i),
        "xc_cross_section_vjp": ([vp, C.POINTER(XcCondition), st, C.POINTER(XcGrid), C.POINTER(XcOpts), vp,
                                  vp, vp, vp, vp, vp, vp, i, vp], i),
        "xc_cross_section_vjp_broadening": ([vp, C.POINTER(XcCondition), st, C.POINTER(XcGrid),
                                             C.POINTER(XcOpts), vp, vp, vp, vp, vp, vp, vp, i, vp], i),
        "xc_set_timing": ([vp, i], i), "xc_last_timings": ([vp, vp], i),
        "xc_last_launch_count": ([vp, C.POINTER(C.c_int64)], i),
        "xc_get_tuning": ([vp, C.c_char_p, st], i),
        "xc_set_tile_shape": ([vp, i, i], i),
        "xc_set_broadening": ([vp, vp, i, vp, i, vp], i),
        "xc_last_sweep_kernels": ([vp, vp, C.POINTER(C.c_int64)], i),
        "xc_count_far_evals": ([vp, C.POINTER(XcCondition), st, C.POINTER(XcGrid), C.POINTER(XcOpts),
                                C.POINTER(C.c_int64), vp], i),
        "xc_cross_section_batched_static": ([C.POINTER(XcLines), st, vp, vp, st, C.POINTER(XcCondition), st,
                                             C.POINTER(XcGrid), C.POINTER(XcOpts), vp, vp], i),
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise XcError(status, lib().xc_last_error().decode())


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, mem) of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (XC_MEM_DEVICE if a.is_cuda else XC_MEM_HOST)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, XC_MEM_HOST


def _stream_of(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def make_condition(T: float, P: float, Q: float = 0.0, dQdT: float = 0.0, mass_da: float = 18.0,
                   T_ref: float = 296.0, P_ref: float = 1.0, gamma_scale: float = 1.0, n_shift: float = 0.0,
                   abundance: float = 1.0) -> XcCondition:
    return XcCondition(T, P, Q, dQdT, mass_da, T_ref, P_ref, gamma_scale, n_shift, abundance)


def make_grid(nu_A: float, step: float, n: int) -> XcGrid:
    return XcGrid(float(nu_A), float(step), int(n))


XC_OPT_NO_TENSOR_CORES = 1


def make_opts(profile: str = "voigt_w4", precision: str = "fp64", cutoff: float = 25.0,
              width_mult: float = 0.0, n_gh: int = 20, tensor_cores: bool = True,
              quantity: str = "absorption", threshold=None, vv_split: float = 0.0, vv_beta: bool = False,
              vv_norm: bool = False) -> XcOpts:
    """tensor_cores=False keeps the FP32 Voigt w4 far wings on the CUDA cores.
    quantity: "absorption" (Eq. e:int) or "emission" (Eq. e:emiss, times h c nu).
    threshold: None, ("constant", I_cut) or ("hitran", nu_crit, I_crit).
    vv_*: the Vectorized Voigt ("voigt_vv"): exact-zone half-width (0: 4 cm^-1), continuity
    factor beta, VVN area normalisation."""
    mode, I_cut, nu_crit, I_crit = 0, 0.0, 0.0, 0.0
    if threshold is not None:
        mode = THRESHOLDS[threshold[0]]
        if mode == 1:
            I_cut = float(threshold[1])
        else:
            nu_crit, I_crit = float(threshold[1]), float(threshold[2])
    return XcOpts(PROFILES[profile], PRECISIONS[precision], float(cutoff), float(width_mult), int(n_gh),
                  0 if tensor_cores else XC_OPT_NO_TENSOR_CORES, QUANTITIES[quantity], mode, I_cut, nu_crit, I_crit,
                  float(vv_split), (1 if vv_beta else 0) | (2 if vv_norm else 0))


_LINE_FIELDS = [("nu", np.float64), ("elower", np.float32), ("A", np.float32), ("gamma_ref", np.float32),
                ("n_T", np.float32), ("g_up", np.int16), ("j_lo", np.int16)]


def partition_function(E, g, T):
    """Q(T) and dQ/dT on the device (Eq. e:pf).  Host numpy in -> numpy out, or CUDA tensors."""
    T_is_dev = _is_torch(T) and T.is_cuda
    if T_is_dev:
        import torch
        Q = torch.empty_like(T)
        dQ = torch.empty_like(T)
        pE, _ = _ptr(E)
        pg, _ = _ptr(g)
        _check(lib().xc_partition_function(pE, pg, len(E), T.data_ptr(), T.numel(), Q.data_ptr(), dQ.data_ptr(),
                                           XC_MEM_DEVICE, _stream_of(T)))
        return Q, dQ
    E = np.ascontiguousarray(E, np.float64)
    g = np.ascontiguousarray(g, np.int32)
    T = np.ascontiguousarray(np.atleast_1d(T), np.float64)
    Q = np.zeros_like(T)
    dQ = np.zeros_like(T)
    _check(lib().xc_partition_function(E.ctypes.data, g.ctypes.data, len(E), T.ctypes.data, len(T), Q.ctypes.data,
                                       dQ.ctypes.data, XC_MEM_HOST, None))
    return Q, dQ


class Engine:
    """One libxc handle on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        _check(lib().xc_create(C.byref(self._h), int(device)))
        self.device = device

    def close(self):
        if self._h:
            lib().xc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- data
    def load_lines(self, lines: Dict[str, object], assume_sorted: bool = False):
        """Copy and sort a line list (dict of numpy arrays or CUDA tensors, 28 B/line)."""
        ptrs, mem = {}, None
        n = len(lines["nu"])
        for k, dt in _LINE_FIELDS:
            a = lines.get(k)
            if a is None:
                ptrs[k] = None
                continue
            if not _is_torch(a):
                a = np.ascontiguousarray(a, dt)
                lines = dict(lines)
                lines[k] = a
            p, m = _ptr(a)
            if mem is None:
                mem = m
            elif m != mem:
                raise ValueError("all line arrays must live in the same memory")
            ptrs[k] = p
        self._keep = lines
        L = XcLines(ptrs["nu"], ptrs["elower"], ptrs["A"], ptrs["gamma_ref"], ptrs["n_T"], ptrs["g_up"],
                    ptrs["j_lo"], mem if mem is not None else XC_MEM_HOST)
        _check(lib().xc_load_lines(self._h, C.byref(L), n, 1 if assume_sorted else 0,
                                   _stream_of(*[lines.get(k) for k, _ in _LINE_FIELDS])))
        self._keep = None

    def num_lines(self) -> int:
        n = C.c_size_t()
        _check(lib().xc_num_lines(self._h, C.byref(n)))
        return n.value

    def get_lines(self) -> Dict[str, np.ndarray]:
        n = self.num_lines()
        out = {k: np.empty(n, dt) for k, dt in _LINE_FIELDS}
        _check(lib().xc_get_lines(self._h, *[out[k].ctypes.data for k, _ in _LINE_FIELDS], XC_MEM_HOST, None))
        return out

    def get_permutation(self) -> np.ndarray:
        out = np.empty(self.num_lines(), np.uint32)
        _check(lib().xc_get_permutation(self._h, out.ctypes.data, XC_MEM_HOST, None))
        return out

    def set_states(self, E, g):
        E = np.ascontiguousarray(E, np.float64)
        g = np.ascontiguousarray(g, np.int32)
        _check(lib().xc_set_states(self._h, E.ctypes.data, g.ctypes.data, len(E), XC_MEM_HOST, None))

    def set_broadening(self, broadeners, j_up=None):
        """Lorentz widths from a mixture of .broad broadeners (make_broadener); j_up: J' of every
        line in load order (needed by a1 tables).  An empty list returns to the lines' widths."""
        arr = (XcBroadener * max(1, len(broadeners)))(*broadeners)
        ju = None if j_up is None else np.ascontiguousarray(j_up, np.int16)
        _check(lib().xc_set_broadening(self._h, C.cast(arr, C.c_void_p), len(broadeners),
                                       None if ju is None else ju.ctypes.data, XC_MEM_HOST, None))

    # ---------------------------------------------------------------- compute
    def line_params(self, cond: XcCondition):
        n = self.num_lines()
        I, a, g = np.empty(n), np.empty(n), np.empty(n)
        _check(lib().xc_line_params(self._h, C.byref(cond), I.ctypes.data, a.ctypes.data, g.ctypes.data,
                                    XC_MEM_HOST, None))
        return I, a, g

    def line_params_device(self, cond: XcCondition, I, alpha, gamma):
        """FP64 I, alpha_D, gamma_L of every (sorted) line into CUDA tensors of n_lines doubles."""
        _check(lib().xc_line_params(self._h, C.byref(cond), I.data_ptr(), alpha.data_ptr(), gamma.data_ptr(),
                                    XC_MEM_DEVICE, _stream_of(I)))

    def count_evals(self, conds: Sequence[XcCondition], grid: XcGrid, opts: XcOpts) -> int:
        arr = (XcCondition * len(conds))(*conds)
        out = C.c_int64()
        _check(lib().xc_count_evals(self._h, arr, len(conds), C.byref(grid), C.byref(opts), C.byref(out), None))
        return out.value

    def cross_section(self, cond: XcCondition, grid: XcGrid, opts: XcOpts, out=None):
        return self.cross_section_batched([cond], grid, opts, out)[0] if out is None else \
            self.cross_section_batched([cond], grid, opts, out)

    def cross_section_batched(self, conds: Sequence[XcCondition], grid: XcGrid, opts: XcOpts, out=None):
        """sigma[n_cond][grid.n] (float64).  out: None (host numpy), numpy, or a CUDA tensor."""
        nc = len(conds)
        arr = (XcCondition * nc)(*conds)
        if out is None:
            out = np.zeros((nc, grid.n), np.float64)
        p, mem = _ptr(out)
        _check(lib().xc_cross_section_batched(self._h, arr, nc, C.byref(grid), C.byref(opts), p, mem,
                                              _stream_of(out)))
        return out

    def cross_section_vjp(self, conds: Sequence[XcCondition], grid: XcGrid, opts: XcOpts, grad_sigma,
                          per_line: bool = True):
        nc = len(conds)
        arr = (XcCondition * nc)(*conds)
        if _is_torch(grad_sigma) and grad_sigma.is_cuda:
            import torch
            dev = grad_sigma.device
            dT = torch.zeros(nc, dtype=torch.float64, device=dev)
            dP = torch.zeros(nc, dtype=torch.float64, device=dev)
            ds = torch.zeros(1, dtype=torch.float64, device=dev)
            dn = torch.zeros(1, dtype=torch.float64, device=dev)
            n = self.num_lines()
            dgl = torch.zeros(n, dtype=torch.float64, device=dev) if per_line else None
            dnl = torch.zeros(n, dtype=torch.float64, device=dev) if per_line else None
            mem = XC_MEM_DEVICE
        else:
            grad_sigma = np.ascontiguousarray(grad_sigma, np.float64)
            dT, dP, ds, dn = np.zeros(nc), np.zeros(nc), np.zeros(1), np.zeros(1)
            n = self.num_lines()
            dgl = np.zeros(n) if per_line else None
            dnl = np.zeros(n) if per_line else None
            mem = XC_MEM_HOST
        P = lambda a: None if a is None else _ptr(a)[0]
        _check(lib().xc_cross_section_vjp(self._h, arr, nc, C.byref(grid), C.byref(opts), P(grad_sigma), P(dT),
                                          P(dP), P(ds), P(dn), P(dgl), P(dnl), mem, _stream_of(grad_sigma)))
        return {"dT": dT, "dP": dP, "d_gamma_scale": ds, "d_n_shift": dn, "d_gamma_ref_line": dgl,
                "d_n_line": dnl}

    def cross_section_vjp_broadening(self, conds: Sequence[XcCondition], grid: XcGrid, opts: XcOpts, grad_sigma,
                                     n_broadeners: int):
        """The adjoint under the handle's broadener mixture: dT, dP, d_gamma_scale, d_n_shift and
        per broadener d_gamma0_broad (a factor on its gamma_0 values) and d_n_broad (a shift of
        its n values).  Device outputs for a CUDA grad_sigma, host numpy otherwise."""
        nc = len(conds)
        arr = (XcCondition * nc)(*conds)
        if _is_torch(grad_sigma) and grad_sigma.is_cuda:
            import torch
            z = lambda m: torch.zeros(m, dtype=torch.float64, device=grad_sigma.device)
            mem = XC_MEM_DEVICE
        else:
            grad_sigma = np.ascontiguousarray(grad_sigma, np.float64)
            z = np.zeros
            mem = XC_MEM_HOST
        out = {"dT": z(nc), "dP": z(nc), "d_gamma_scale": z(1), "d_n_shift": z(1),
               "d_gamma0_broad": z(n_broadeners), "d_n_broad": z(n_broadeners)}
        P = lambda a: _ptr(a)[0]
        _check(lib().xc_cross_section_vjp_broadening(self._h, arr, nc, C.byref(grid), C.byref(opts), P(grad_sigma),
                                                     P(out["dT"]), P(out["dP"]), P(out["d_gamma_scale"]),
                                                     P(out["d_n_shift"]), P(out["d_gamma0_broad"]),
                                                     P(out["d_n_broad"]), mem, _stream_of(grad_sigma)))
        return out

    # ---------------------------------------------------------------- accounting
    def set_timing(self, on: bool = True):
        _check(lib().xc_set_timing(self._h, 1 if on else 0))

    def timings(self) -> Dict[str, float]:
        ms = (C.c_float * 8)()
        _check(lib().xc_last_timings(self._h, ms))
        names = ["sort", "gather", "Q", "params_or_sweep", "ranges_or_core", "profile", "vjp", "copies"]
        return {k: float(v) for k, v in zip(names, ms)}

    def set_tile_shape(self, R: int = 0, CG: int = 0):
        """Fix the FP32 CUDA-core kernel's tile shape (R points per thread, CG conditions
        per tile); (0, 0) returns to the autotuner."""
        _check(lib().xc_set_tile_shape(self._h, int(R), int(CG)))

    def sweep_kernels(self):
        """(far-wing tensor-core ms, CUDA-core kernel ms, centre-zone ms, MMA count) of the
        last timed FP32 batched call; -1 for a kernel that did not run."""
        ms = (C.c_double * 3)()
        mma = C.c_int64()
        _check(lib().xc_last_sweep_kernels(self._h, ms, C.byref(mma)))
        return ms[0], ms[1], ms[2], int(mma.value)

    def count_far_evals(self, conds: Sequence[XcCondition], grid: XcGrid, opts: XcOpts) -> int:
        """(line, point, condition) evaluations the tensor-core far-wing kernel takes in a
        batched call with these arguments (0 when it would not run)."""
        arr = (XcCondition * len(conds))(*conds)
        v = C.c_int64()
        _check(lib().xc_count_far_evals(self._h, arr, len(conds), C.byref(grid), C.byref(opts), C.byref(v), None))
        return int(v.value)

    def tuning(self) -> str:
        buf = C.create_string_buffer(4096)
        _check(lib().xc_get_tuning(self._h, buf, 4096))
        return buf.value.decode()

    def last_launch_count(self) -> int:
        v = C.c_int64()
        _check(lib().xc_last_launch_count(self._h, C.byref(v)))
        return v.value


# ---------------------------------------------------------------------------- autograd
def cross_section_autograd(engine: "Engine", T, P, gamma_scale, n_shift, grid: XcGrid, opts: XcOpts,
                           mass_da: float = 18.0, T_ref: float = 296.0, P_ref: float = 1.0):
    """Differentiable batched cross section: sigma[C][N] as a function of the tensors
    T[C], P[C] and the scalars gamma_scale, n_shift (float64 tensors).  The backward
    pass calls the library's adjoint (xc_cross_section_vjp)."""
    import torch

    class _CrossSection(torch.autograd.Function):
        @staticmethod
        def forward(ctx, T_, P_, s_, n_):
            conds = [make_condition(float(t), float(p), mass_da=mass_da, T_ref=T_ref, P_ref=P_ref,
                                    gamma_scale=float(s_), n_shift=float(n_))
                     for t, p in zip(T_.detach().cpu().tolist(), P_.detach().cpu().tolist())]
            ctx.conds = conds
            out = torch.empty((len(conds), grid.n), dtype=torch.float64, device=f"cuda:{engine.device}")
            engine.cross_section_batched(conds, grid, opts, out)
            return out

        @staticmethod
        def backward(ctx, g):
            r = engine.cross_section_vjp(ctx.conds, grid, opts, g.contiguous().to(torch.float64),
                                         per_line=False)
            dT = r["dT"].to(T.device)
            dP = r["dP"].to(P.device)
            ds = r["d_gamma_scale"].reshape(()).to(torch.as_tensor(gamma_scale).device)
            dn = r["d_n_shift"].reshape(()).to(torch.as_tensor(n_shift).device)
            return dT, dP, ds, dn

    return _CrossSection.apply(T, P, gamma_scale, n_shift)
