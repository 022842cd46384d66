"""FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, obviously correct
restatement of the ExoCross cross-section method in C (``xo.c``), loaded
through ctypes.  It shares no code with the CUDA library; both only consume
inputs from :mod:`xcsynth`.

Functions follow the paper's equations (arXiv:1801.09803):
Eq. (e:pf) partition function, Eq. (e:int) intensity, Eq. (e:alphaD) Doppler
HWHM, Eq. (e:gamma_L) Lorentz HWHM, Eqs. (e:Gauss), (e:lor), (e:Voigt) profiles,
Humlicek's w4 for the Voigt function, Eqs. (e:V-quad) and (e:sigma:quad) for
Gauss-Hermite Voigt, Eqs. (eqn:sig_ij) and (eqn:sig_lor-2) for the binned
Gaussian and Lorentzian, and the sampling method of Sec. 3.1.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xo.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROFILES = {"doppler": 0, "lorentz": 1, "voigt_w4": 2, "voigt_gh_binned": 3, "voigt_gh_sampled": 4,
            "doppler_binned": 5, "lorentz_binned": 6, "voigt_vv": 7}


class Condition(C.Structure):
    _fields_ = [("T", C.c_double), ("P", C.c_double), ("Q", C.c_double), ("dQdT", C.c_double),
                ("mass_da", C.c_double), ("T_ref", C.c_double), ("P_ref", C.c_double),
                ("gamma_scale", C.c_double), ("n_shift", C.c_double), ("abundance", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("profile", C.c_int), ("cutoff", C.c_double), ("width_mult", C.c_double),
                ("n_gh", C.c_int), ("quantity", C.c_int), ("thr_mode", C.c_int), ("I_cut", C.c_double),
                ("nu_crit", C.c_double), ("I_crit", C.c_double), ("vv_split", C.c_double), ("vv_beta", C.c_int),
                ("vv_norm", C.c_int)]


QUANTITIES = {"absorption": 0, "emission": 1}


class Broadener(C.Structure):
    _fields_ = [("type", C.c_int), ("fraction", C.c_double), ("gamma0", C.c_double), ("n", C.c_double),
                ("n_entries", C.c_longlong), ("j_lo", C.c_void_p), ("j_up", C.c_void_p),
                ("gamma0_j", C.c_void_p), ("n_j", C.c_void_p)]


BROAD_TYPES = {"constant": 0, "a0": 1, "a1": 2}


def make_broadener(kind: str, fraction: float, gamma0: float, n: float, table=None) -> Broadener:
    """One broadener: kind "constant", "a0" (table {J'': (gamma0, n)}) or "a1" (table
    {(J'', J'): (gamma0, n)}); gamma0 / n are the defaults for lines the table does not list."""
    t = BROAD_TYPES[kind]
    rows = sorted((table or {}).items())
    jl = np.array([k if t == 1 else k[0] for k, _ in rows], np.int32)
    ju = np.array([k[1] for k, _ in rows] if t == 2 else [], np.int32)
    g0 = np.array([v[0] for _, v in rows], np.float64)
    nn = np.array([v[1] for _, v in rows], np.float64)
    b = Broadener(t, float(fraction), float(gamma0), float(n), len(rows), _p(jl), _p(ju) if t == 2 else None,
                  _p(g0), _p(nn))
    b._keep = (jl, ju, g0, nn)   # the arrays the pointers refer to
    return b


def _broad_array(broadeners):
    arr = (Broadener * len(broadeners))(*broadeners)
    return arr


def build(force: bool = False) -> str:
    """Compile xo.c into liboracle.so (plain gcc; OpenMP for the threaded baseline)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        L.xo_c2.restype = d
        L.xo_partition_function.argtypes = [vp, vp, C.c_size_t, d, vp, vp]
        L.xo_intensity.argtypes = [d, d, d, d, C.POINTER(Condition)]
        L.xo_emissivity.argtypes = [d, d, d, d, C.POINTER(Condition)]
        L.xo_emissivity.restype = d
        L.xo_threshold.argtypes = [d, d, C.POINTER(Opts)]
        L.xo_threshold.restype = d
        L.xo_voigt_vv.argtypes = [d, d, d, d, d, i]
        L.xo_voigt_vv.restype = d
        L.xo_gamma_mixture.argtypes = [i, i, vp, i, C.POINTER(Condition)]
        L.xo_gamma_mixture.restype = d
        L.xo_cross_section_broad.argtypes = [vp] * 6 + [C.c_size_t, vp, i, C.POINTER(Condition), d, d,
                                                        C.c_longlong, C.POINTER(Opts), vp, i]
        L.xo_cross_section_broad.restype = i
        L.xo_intensity.restype = d
        L.xo_alpha_doppler.argtypes = [d, C.POINTER(Condition)]
        L.xo_alpha_doppler.restype = d
        L.xo_gamma_lorentz.argtypes = [d, d, C.POINTER(Condition)]
        L.xo_gamma_lorentz.restype = d
        L.xo_w4_deriv.argtypes = [d, d, vp, vp, vp, vp]
        L.xo_gauss_hermite.argtypes = [i, vp, vp]
        L.xo_gauss_hermite.restype = i
        for f in ("xo_gauss", "xo_lorentz"):
            getattr(L, f).argtypes = [d, d]
            getattr(L, f).restype = d
        L.xo_voigt_w4.argtypes = [d, d, d]
        L.xo_voigt_w4.restype = d
        L.xo_voigt_gh.argtypes = [d, d, d, i, vp, vp]
        L.xo_voigt_gh.restype = d
        L.xo_voigt_gh_binned.argtypes = [d, d, d, d, i, vp, vp]
        L.xo_voigt_gh_binned.restype = d
        for f in ("xo_gauss_binned", "xo_lorentz_binned"):
            getattr(L, f).argtypes = [d, d, d]
            getattr(L, f).restype = d
        L.xo_profile.argtypes = [i, d, d, d, d, i, vp, vp, vp, vp]
        L.xo_profile.restype = d
        L.xo_cross_section.argtypes = [vp] * 6 + [C.c_size_t, C.POINTER(Condition), d, d, C.c_longlong,
                                                   C.POINTER(Opts), vp, i]
        L.xo_cross_section.restype = i
        L.xo_cross_section_points.argtypes = [vp] * 6 + [C.c_size_t, C.POINTER(Condition), d, d, vp,
                                                          C.c_longlong, C.POINTER(Opts), vp, i]
        L.xo_cross_section_points.restype = i
        L.xo_count_evals.argtypes = [vp, vp, vp, C.c_size_t, C.POINTER(Condition), d, d, C.c_longlong,
                                     C.POINTER(Opts)]
        L.xo_count_evals.restype = C.c_longlong
        L.xo_cross_section_vjp.argtypes = [vp] * 6 + [C.c_size_t, C.POINTER(Condition), i, d, d,
                                                       C.c_longlong, C.POINTER(Opts), vp,
                                                       vp, vp, vp, vp, vp, vp]
        L.xo_cross_section_vjp.restype = i
        L.xo_cross_section_vjp_broad.argtypes = [vp] * 6 + [C.c_size_t, vp, i, C.POINTER(Condition), i, d, d,
                                                             C.c_longlong, C.POINTER(Opts), vp,
                                                             vp, vp, vp, vp, vp, vp]
        L.xo_cross_section_vjp_broad.restype = i
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def c2() -> float:
    """Second radiation constant hc/k_B in cm K (CODATA 2018 exact values)."""
    return lib().xo_c2()


def partition_function(E: np.ndarray, g: np.ndarray, T: float):
    """Eq. (e:pf): Q(T) = sum_n g_n exp(-c2 E_n / T), and dQ/dT."""
    E = np.ascontiguousarray(E, np.float64)
    g = np.ascontiguousarray(g, np.int32)
    q, dq = np.zeros(1), np.zeros(1)
    lib().xo_partition_function(_p(E), _p(g), len(E), float(T), _p(q), _p(dq))
    return float(q[0]), float(dq[0])


def make_condition(T: float, P: float, Q: float, dQdT: float = 0.0, mass_da: float = 18.0,
                   T_ref: float = 296.0, P_ref: float = 1.0, gamma_scale: float = 1.0,
                   n_shift: float = 0.0, abundance: float = 1.0) -> Condition:
    return Condition(T, P, Q, dQdT, mass_da, T_ref, P_ref, gamma_scale, n_shift, abundance)


def make_opts(profile: str = "voigt_w4", cutoff: float = 25.0, width_mult: float = 0.0,
              n_gh: int = 20, quantity: str = "absorption", threshold=None, vv_split: float = 4.0,
              vv_beta: bool = False, vv_norm: bool = False) -> Opts:
    """threshold: None, ("constant", I_cut) or ("hitran", nu_crit, I_crit).  vv_*: the
    Vectorized Voigt ("voigt_vv"): exact zone, continuity factor beta, VVN normalisation."""
    mode, I_cut, nu_crit, I_crit = 0, 0.0, 0.0, 0.0
    if threshold is not None:
        if threshold[0] == "constant":
            mode, I_cut = 1, float(threshold[1])
        elif threshold[0] == "hitran":
            mode, nu_crit, I_crit = 2, float(threshold[1]), float(threshold[2])
        else:
            raise ValueError(f"unknown threshold {threshold[0]!r}")
    return Opts(PROFILES[profile], cutoff, width_mult, n_gh, QUANTITIES[quantity], mode, I_cut, nu_crit, I_crit,
                float(vv_split), int(bool(vv_beta)), int(bool(vv_norm)))


def intensity(nu, elower, A, g_up, cond: Condition) -> float:
    return lib().xo_intensity(float(nu), float(elower), float(A), float(g_up), C.byref(cond))


def emissivity(nu, elower, A, g_up, cond: Condition) -> float:
    """Eq. (e:emiss) times the photon energy h c nu: erg/s/sr per molecule."""
    return lib().xo_emissivity(float(nu), float(elower), float(A), float(g_up), C.byref(cond))


def voigt_vv(D, alpha, gamma, nu_l, split=4.0, beta=False):
    """Eq. (e:fast-v): Vectorized Voigt of a line at nu_l."""
    return lib().xo_voigt_vv(float(D), float(alpha), float(gamma), float(nu_l), float(split), int(bool(beta)))


def gamma_mixture(j_lo, j_up, broadeners, cond: Condition) -> float:
    """Lorentz HWHM of a line with these J under a mixture of broadeners."""
    arr = _broad_array(broadeners)
    return lib().xo_gamma_mixture(int(j_lo), int(j_up), C.cast(arr, C.c_void_p), len(broadeners), C.byref(cond))


def cross_section_broad(lines, j_up, broadeners, cond: Condition, nu_A, step, n_pts, opts: Opts,
                        nthreads: Optional[int] = None) -> np.ndarray:
    """Cross section with every line's Lorentz HWHM from the broadener mixture (J'' from
    lines["j_lo"], J' from j_up)."""
    nu = np.ascontiguousarray(lines["nu"], np.float64)
    el = np.ascontiguousarray(lines["elower"], np.float32)
    A = np.ascontiguousarray(lines["A"], np.float32)
    jl = np.ascontiguousarray(lines["j_lo"], np.int16)
    ju = np.ascontiguousarray(j_up, np.int16)
    g = np.ascontiguousarray(lines["g_up"], np.int16)
    out = np.zeros(max(int(n_pts), 0))
    arr = _broad_array(broadeners)
    nt = nthreads or min(16, os.cpu_count() or 1)
    rc = lib().xo_cross_section_broad(_p(nu), _p(el), _p(A), _p(jl), _p(ju), _p(g), len(nu), C.cast(arr, C.c_void_p),
                                      len(broadeners), C.byref(cond), float(nu_A), float(step), int(n_pts),
                                      C.byref(opts), _p(out), int(nt))
    if rc != 0:
        raise RuntimeError(f"xo_cross_section_broad failed: {rc}")
    return out


def threshold(nu, T, opts: Opts) -> float:
    """The intensity threshold at nu (0 when opts sets none)."""
    return lib().xo_threshold(float(nu), float(T), C.byref(opts))


def alpha_doppler(nu, cond: Condition) -> float:
    return lib().xo_alpha_doppler(float(nu), C.byref(cond))


def gamma_lorentz(gamma_ref, n_T, cond: Condition) -> float:
    return lib().xo_gamma_lorentz(float(gamma_ref), float(n_T), C.byref(cond))


def w4(x: float, y: float, deriv: bool = False):
    """Humlicek w4 value (complex) and optionally its derivative dF/dt, t = y - ix."""
    a = np.zeros(4)
    lib().xo_w4_deriv(float(x), float(y), _p(a[0:1]), _p(a[1:2]), _p(a[2:3]), _p(a[3:4]))
    w = complex(a[0], a[1])
    return (w, complex(a[2], a[3])) if deriv else w


def gauss_hermite(n: int):
    x, w = np.zeros(n), np.zeros(n)
    rc = lib().xo_gauss_hermite(int(n), _p(x), _p(w))
    if rc != 0:
        raise RuntimeError(f"xo_gauss_hermite({n}) failed: {rc}")
    return x, w


def gauss(D, alpha):
    return lib().xo_gauss(float(D), float(alpha))


def lorentz(D, gamma):
    return lib().xo_lorentz(float(D), float(gamma))


def voigt_w4(D, alpha, gamma):
    return lib().xo_voigt_w4(float(D), float(alpha), float(gamma))


def voigt_gh(D, alpha, gamma, n=20):
    x, w = gauss_hermite(n)
    return lib().xo_voigt_gh(float(D), float(alpha), float(gamma), n, _p(x), _p(w))


def voigt_gh_binned(D, h, alpha, gamma, n=20):
    x, w = gauss_hermite(n)
    return lib().xo_voigt_gh_binned(float(D), float(h), float(alpha), float(gamma), n, _p(x), _p(w))


def gauss_binned(D, h, alpha):
    """Eq. (eqn:sig_ij) without I: the Gaussian averaged over the bin [D - h/2, D + h/2]."""
    return lib().xo_gauss_binned(float(D), float(h), float(alpha))


def lorentz_binned(D, h, gamma):
    """Eq. (eqn:sig_lor-2) without I: the Lorentzian averaged over the bin [D - h/2, D + h/2]."""
    return lib().xo_lorentz_binned(float(D), float(h), float(gamma))


def profile(name: str, D, h, alpha, gamma, n_gh=20):
    """Profile value with dV/dalpha and dV/dgamma."""
    x, w = gauss_hermite(n_gh)
    da, dg = np.zeros(1), np.zeros(1)
    v = lib().xo_profile(PROFILES[name], float(D), float(h), float(alpha), float(gamma), n_gh,
                         _p(x), _p(w), _p(da), _p(dg))
    return v, float(da[0]), float(dg[0])


def _line_arrays(lines: Dict[str, np.ndarray]):
    return (np.ascontiguousarray(lines["nu"], np.float64),
            np.ascontiguousarray(lines["elower"], np.float32),
            np.ascontiguousarray(lines["A"], np.float32),
            np.ascontiguousarray(lines["gamma_ref"], np.float32),
            np.ascontiguousarray(lines["n_T"], np.float32),
            np.ascontiguousarray(lines["g_up"], np.int16))


def cross_section(lines: Dict[str, np.ndarray], cond: Condition, nu_A: float, step: float,
                  n_pts: int, opts: Opts, nthreads: int = 1) -> np.ndarray:
    """sigma_k = sum_l I_l f(nu_k - nu_l) over |nu_k - nu_l| <= cut (Sec. 3.1 sampling)."""
    arrs = _line_arrays(lines)
    out = np.zeros(int(n_pts), np.float64)
    rc = lib().xo_cross_section(*[_p(a) for a in arrs], len(arrs[0]), C.byref(cond), float(nu_A),
                                float(step), int(n_pts), C.byref(opts), _p(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"xo_cross_section failed: {rc}")
    return out


def cross_section_points(lines_sorted: Dict[str, np.ndarray], cond: Condition, nu_A: float, step: float,
                         k_list, opts: Opts, nthreads: int = 1) -> np.ndarray:
    """sigma at the grid points k_list, one point at a time (lines must be sorted by nu)."""
    arrs = _line_arrays(lines_sorted)
    ks = np.ascontiguousarray(k_list, np.int64)
    out = np.zeros(len(ks), np.float64)
    rc = lib().xo_cross_section_points(*[_p(a) for a in arrs], len(arrs[0]), C.byref(cond), float(nu_A),
                                       float(step), _p(ks), len(ks), C.byref(opts), _p(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"xo_cross_section_points failed: {rc}")
    return out


def count_evals(lines, cond: Condition, nu_A, step, n_pts, opts: Opts) -> int:
    arrs = _line_arrays(lines)
    return int(lib().xo_count_evals(_p(arrs[0]), _p(arrs[3]), _p(arrs[4]), len(arrs[0]),
                                    C.byref(cond), float(nu_A), float(step), int(n_pts),
                                    C.byref(opts)))


def cross_section_vjp(lines, conds: Sequence[Condition], nu_A, step, n_pts, opts: Opts,
                      grad_sigma: np.ndarray, per_line: bool = True):
    arrs = _line_arrays(lines)
    nc = len(conds)
    carr = (Condition * nc)(*conds)
    g = np.ascontiguousarray(grad_sigma, np.float64).reshape(nc, int(n_pts))
    dT, dP = np.zeros(nc), np.zeros(nc)
    dgs, dns = np.zeros(1), np.zeros(1)
    n = len(arrs[0])
    dgl = np.zeros(n) if per_line else None
    dnl = np.zeros(n) if per_line else None
    rc = lib().xo_cross_section_vjp(*[_p(a) for a in arrs], n, carr, nc, float(nu_A), float(step),
                                    int(n_pts), C.byref(opts), _p(g), _p(dT), _p(dP), _p(dgs),
                                    _p(dns), _p(dgl), _p(dnl))
    if rc != 0:
        raise RuntimeError(f"xo_cross_section_vjp failed: {rc}")
    return {"dT": dT, "dP": dP, "d_gamma_scale": float(dgs[0]), "d_n_shift": float(dns[0]),
            "d_gamma_ref_line": dgl, "d_n_line": dnl}


def cross_section_vjp_broad(lines, j_up, broadeners, conds: Sequence[Condition], nu_A, step, n_pts, opts: Opts,
                            grad_sigma: np.ndarray):
    """The adjoint with every line's Lorentz HWHM from the broadener mixture: dT, dP per
    condition, d_gamma_scale, d_n_shift, and per broadener d_gamma0 (dL/d of a scale on all
    its gamma_0 values, at 1) and d_n (dL/d of a shift of all its n values, at 0)."""
    nu = np.ascontiguousarray(lines["nu"], np.float64)
    el = np.ascontiguousarray(lines["elower"], np.float32)
    A = np.ascontiguousarray(lines["A"], np.float32)
    jl = np.ascontiguousarray(lines["j_lo"], np.int16)
    ju = np.ascontiguousarray(j_up, np.int16)
    g = np.ascontiguousarray(lines["g_up"], np.int16)
    nc, nb = len(conds), len(broadeners)
    carr = (Condition * nc)(*conds)
    arr = _broad_array(broadeners)
    gs = np.ascontiguousarray(grad_sigma, np.float64).reshape(nc, int(n_pts))
    dT, dP, dgs, dns = np.zeros(nc), np.zeros(nc), np.zeros(1), np.zeros(1)
    dg0, dnb = np.zeros(nb), np.zeros(nb)
    rc = lib().xo_cross_section_vjp_broad(_p(nu), _p(el), _p(A), _p(jl), _p(ju), _p(g), len(nu),
                                          C.cast(arr, C.c_void_p), nb, carr, nc, float(nu_A), float(step),
                                          int(n_pts), C.byref(opts), _p(gs), _p(dT), _p(dP), _p(dgs), _p(dns),
                                          _p(dg0), _p(dnb))
    if rc != 0:
        raise RuntimeError(f"xo_cross_section_vjp_broad failed: {rc}")
    return {"dT": dT, "dP": dP, "d_gamma_scale": float(dgs[0]), "d_n_shift": float(dns[0]),
            "d_gamma0_broad": dg0, "d_n_broad": dnb}
