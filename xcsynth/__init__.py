"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module only *makes inputs*: line lists, state lists, (T, P) condition
sets and grid/workload descriptions.  It contains none of the cross-section
arithmetic (no intensities, widths or profiles), so both sides can use it
without sharing any of the method.

Counter-based generator
-----------------------
Every random field of record ``i`` comes from a stateless hash of
``(seed, i, field)``, so line ``i`` is the same line whatever slice of the
list is generated, on whatever device.  The hash is the SplitMix64 output
function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), applied to ``seed XOR ((8*i + field) * 0x9E3779B97F4A7C15)``
modulo 2**64; the top 53 bits give a uniform double in [0, 1).

Line-list recipe (values the method's paper leaves open are fixed here):

* nu    : uniform on the half-open interval (lo, hi], drawn as hi - U*(hi-lo),
          so nu > 0 always (nu = 0 would make the intensity infinite).
* E''   : exponential with scale 3000 cm^-1, then clamped to 20000 (a clamp,
          not a redraw).
* J''   : uniform integer 0..jmax (jmax = 50).
* J'    : J'' + dJ with dJ uniform in {-1, 0, +1}; dJ = -1 at J'' = 0 becomes +1.
* g'    : g_ns * (2 J' + 1)   (upper-state total degeneracy, int16).
* A     : log10 A uniform in [-6, 2]  (s^-1).
* gamma_ref : uniform in [0.02, 0.1] cm^-1 at T_ref = 296 K, P_ref = 1 bar.
* n     : uniform in [0.4, 0.8].

Storage follows the line record of the GPU library: nu float64; E'', A,
gamma_ref, n float32; g', J'' int16 (28 bytes per line).  Consumers that work
in float64 (the oracle) read the stored float32 values exactly, so both sides
see bit-identical inputs.

State list (for Q(T)): ``n`` states with E from the same clamped exponential,
J uniform 0..jmax and g = g_ns (2J+1), from a separate seed stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

__all__ = [
    "GOLDEN", "uniform_hash", "gen_lines", "gen_states", "Workload",
    "WORKLOADS", "conditions_for", "grid_for", "subset_indices",
]

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STATES_SALT = 0x5354415445530000  # "STATES\0\0"

# field numbers of a line record
F_NU, F_E, F_J, F_DJ, F_A, F_GAMMA, F_N = range(7)
# field numbers of a state record
FS_E, FS_J = 0, 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform_hash(seed: int, idx: np.ndarray, fld: int) -> np.ndarray:
    """Uniform doubles in [0, 1) for records ``idx`` (uint64 array) and one field."""
    with np.errstate(over="ignore"):
        ctr = (idx.astype(np.uint64) * np.uint64(8) + np.uint64(fld)) * GOLDEN
        z = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _exp_clamped(u: np.ndarray, scale: float, cap: float) -> np.ndarray:
    # inverse CDF of the exponential; log1p(-u) is finite because u < 1
    return np.minimum(-scale * np.log1p(-u), cap)


def gen_lines(seed: int, i0: int, n: int, nu_lo: float, nu_hi: float,
              jmax: int = 50, g_ns: int = 1, chunk: int = 1 << 22) -> Dict[str, np.ndarray]:
    """Lines ``i0 .. i0+n-1`` of the seeded synthetic list (unsorted in nu)."""
    out = {
        "nu": np.empty(n, np.float64),
        "elower": np.empty(n, np.float32),
        "A": np.empty(n, np.float32),
        "gamma_ref": np.empty(n, np.float32),
        "n_T": np.empty(n, np.float32),
        "g_up": np.empty(n, np.int16),
        "j_lo": np.empty(n, np.int16),
    }
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(i0 + s, i0 + e, dtype=np.uint64)
        u = uniform_hash(seed, idx, F_NU)
        out["nu"][s:e] = nu_hi - u * (nu_hi - nu_lo)
        out["elower"][s:e] = _exp_clamped(uniform_hash(seed, idx, F_E), 3000.0, 20000.0)
        jl = np.floor(uniform_hash(seed, idx, F_J) * (jmax + 1)).astype(np.int64)
        dj = np.floor(uniform_hash(seed, idx, F_DJ) * 3).astype(np.int64) - 1
        dj = np.where((jl == 0) & (dj == -1), 1, dj)
        ju = jl + dj
        out["j_lo"][s:e] = jl
        out["g_up"][s:e] = g_ns * (2 * ju + 1)
        out["A"][s:e] = np.power(10.0, -6.0 + 8.0 * uniform_hash(seed, idx, F_A))
        out["gamma_ref"][s:e] = 0.02 + 0.08 * uniform_hash(seed, idx, F_GAMMA)
        out["n_T"][s:e] = 0.4 + 0.4 * uniform_hash(seed, idx, F_N)
    return out


def gen_states(seed: int, n: int = 5000, jmax: int = 50, g_ns: int = 1):
    """State list (E float64 cm^-1, g int32) for the partition-function sum."""
    s = (seed ^ _STATES_SALT) & 0xFFFFFFFFFFFFFFFF
    idx = np.arange(n, dtype=np.uint64)
    E = _exp_clamped(uniform_hash(s, idx, FS_E), 3000.0, 20000.0)
    J = np.floor(uniform_hash(s, idx, FS_J) * (jmax + 1)).astype(np.int64)
    g = (g_ns * (2 * J + 1)).astype(np.int32)
    return E.astype(np.float64), g


def subset_indices(n_total: int, n_sub: int, seed: int) -> np.ndarray:
    """A seeded, sorted choice of ``n_sub`` distinct record numbers in [0, n_total)."""
    rng = np.random.default_rng(seed)
    if n_sub >= n_total:
        return np.arange(n_total, dtype=np.int64)
    return np.sort(rng.choice(n_total, size=n_sub, replace=False)).astype(np.int64)


def gen_lines_at(seed: int, idx: np.ndarray, nu_lo: float, nu_hi: float,
                 jmax: int = 50, g_ns: int = 1) -> Dict[str, np.ndarray]:
    """Lines with arbitrary record numbers ``idx`` (same values as gen_lines)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u = uniform_hash(seed, idx, F_NU)
    jl = np.floor(uniform_hash(seed, idx, F_J) * (jmax + 1)).astype(np.int64)
    dj = np.floor(uniform_hash(seed, idx, F_DJ) * 3).astype(np.int64) - 1
    dj = np.where((jl == 0) & (dj == -1), 1, dj)
    return {
        "nu": (nu_hi - u * (nu_hi - nu_lo)).astype(np.float64),
        "elower": _exp_clamped(uniform_hash(seed, idx, F_E), 3000.0, 20000.0).astype(np.float32),
        "A": np.power(10.0, -6.0 + 8.0 * uniform_hash(seed, idx, F_A)).astype(np.float32),
        "gamma_ref": (0.02 + 0.08 * uniform_hash(seed, idx, F_GAMMA)).astype(np.float32),
        "n_T": (0.4 + 0.4 * uniform_hash(seed, idx, F_N)).astype(np.float32),
        "g_up": (g_ns * (2 * (jl + dj) + 1)).astype(np.int16),
        "j_lo": jl.astype(np.int16),
    }


def gen_lines_torch(seed: int, i0: int, n: int, nu_lo: float, nu_hi: float, device="cuda",
                    jmax: int = 50, g_ns: int = 1, chunk: int = 1 << 26):
    """The same lines as gen_lines, generated with torch on `device` (for lists too
    large to build on the host).  uint64 arithmetic is emulated on int64 tensors:
    products wrap modulo 2^64 and right shifts are masked to be logical.  nu, J'',
    J', gamma_ref and n_T are bit-identical to gen_lines; E'' and A go through
    log1p / pow of the device library and can differ from numpy's in the last
    float64 bit before rounding to float32."""
    import torch

    def s64(v):  # uint64 constant as int64
        v &= 0xFFFFFFFFFFFFFFFF
        return v - (1 << 64) if v >= (1 << 63) else v

    m1, m2, gold = s64(0xBF58476D1CE4E5B9), s64(0x94D049BB133111EB), s64(0x9E3779B97F4A7C15)
    sd = s64(seed)

    def lsr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    def uni(idx, fld):
        z = (idx * 8 + fld) * gold
        z = z ^ sd
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        return lsr(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)

    out = {
        "nu": torch.empty(n, dtype=torch.float64, device=device),
        "elower": torch.empty(n, dtype=torch.float32, device=device),
        "A": torch.empty(n, dtype=torch.float32, device=device),
        "gamma_ref": torch.empty(n, dtype=torch.float32, device=device),
        "n_T": torch.empty(n, dtype=torch.float32, device=device),
        "g_up": torch.empty(n, dtype=torch.int16, device=device),
        "j_lo": torch.empty(n, dtype=torch.int16, device=device),
    }
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(i0 + s, i0 + e, dtype=torch.int64, device=device)
        out["nu"][s:e] = nu_hi - uni(idx, F_NU) * (nu_hi - nu_lo)
        out["elower"][s:e] = torch.clamp(-3000.0 * torch.log1p(-uni(idx, F_E)), max=20000.0).to(torch.float32)
        jl = torch.floor(uni(idx, F_J) * (jmax + 1)).to(torch.int64)
        dj = torch.floor(uni(idx, F_DJ) * 3).to(torch.int64) - 1
        dj = torch.where((jl == 0) & (dj == -1), torch.ones_like(dj), dj)
        out["j_lo"][s:e] = jl.to(torch.int16)
        out["g_up"][s:e] = (g_ns * (2 * (jl + dj) + 1)).to(torch.int16)
        out["A"][s:e] = torch.pow(10.0, -6.0 + 8.0 * uni(idx, F_A)).to(torch.float32)
        out["gamma_ref"][s:e] = (0.02 + 0.08 * uni(idx, F_GAMMA)).to(torch.float32)
        out["n_T"][s:e] = (0.4 + 0.4 * uni(idx, F_N)).to(torch.float32)
    return out


# ---------------------------------------------------------------------------
# Workload descriptions (sizes and conditions of the five benchmark cases)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n_lines: int
    nu_lo: float
    nu_hi: float
    grid_lo: float
    grid_hi: float
    step: float
    temperatures: List[float]
    pressures: List[float]
    profile: str = "voigt_w4"
    cutoff: float = 25.0
    cutoff_width_mult: float = 0.0     # >0: per-line cut = min(cutoff, mult*max(alpha, gamma))
    n_gh: int = 20
    mass_da: float = 18.0
    g_ns: int = 1
    n_states: int = 5000
    seed: int = 180109803
    note: str = ""

    @property
    def n_points(self) -> int:
        return int(round((self.grid_hi - self.grid_lo) / self.step)) + 1

    @property
    def n_conditions(self) -> int:
        return len(self.temperatures) * len(self.pressures)


WORKLOADS: Dict[str, Workload] = {
    # plain FP64 method, one condition, 1e5 lines, 200001 points
    "C1": Workload("C1", 100_000, 1000.0, 3000.0, 1000.0, 3000.0, 0.01,
                   [1000.0], [1.0], seed=180109803 + 1),
    # one condition at scale, 1e7 lines, 1 000 001 points, width-limited cut
    "C2": Workload("C2", 10_000_000, 0.0, 10000.0, 0.0, 10000.0, 0.01,
                   [1500.0], [1.0], cutoff_width_mult=500.0, seed=180109803 + 2),
    # 32 conditions in one launch, 1e8 lines, 1 000 001 points
    "C3": Workload("C3", 100_000_000, 0.0, 10000.0, 0.0, 10000.0, 0.01,
                   [300.0 * 10.0 ** (i / 7.0) for i in range(8)],
                   [1e-3, 1e-1, 1.0, 10.0], seed=180109803 + 3),
    # differentiation: C1 generator and grid, 1e7 lines, 2 x 2 conditions
    "C4": Workload("C4", 10_000_000, 1000.0, 3000.0, 1000.0, 3000.0, 0.01,
                   [800.0, 1600.0], [0.1, 1.0], seed=180109803 + 4),
    # mixed precision at maximum size, 1e9 lines, 2 000 001 points
    "C5": Workload("C5", 1_000_000_000, 0.0, 20000.0, 0.0, 20000.0, 0.01,
                   [2000.0], [1.0], seed=180109803 + 5),
}


def conditions_for(w: Workload) -> List[Dict[str, float]]:
    """(T, P) pairs, temperature-major (all pressures of T0, then T1, ...)."""
    return [{"T": float(T), "P": float(P)} for T in w.temperatures for P in w.pressures]


def grid_for(w: Workload) -> Dict[str, float]:
    return {"nu_A": w.grid_lo, "step": w.step, "n": w.n_points}
