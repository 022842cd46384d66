"""The grid partition of one cross section, run through the library on one GPU.

The path shards along the wavenumber grid with no reduction: shard r owns the
contiguous grid range [k0, k1) and needs only the lines within one cutoff of it,
a contiguous range of the sorted list found by binary search (the halo).  Here
the shards of a 4-way partition run one after another, each in its own handle
loaded with its halo range only, through xc_cross_section_batched, and their
concatenation is compared with the unsharded call: bit for bit on the FP64 path
(a grid step of 2^-7 makes every grid point exact in binary, so a shard's own grid
reproduces the same points, and each point sums the same lines in the same order),
and within the FP32 paths' agreement tolerance (2e-5 relative above 1e-6 of each
condition's peak: tile boundaries move with the shard, which changes the FP32
summation order) on the FP32 batched sweep over 16 conditions (far wings on the
tensor cores), with a partial last block in every shard.
"""
import numpy as np
import pytest

import xcsynth as xs
from paper_1801_09803_gb300.shard import grid_shard, halo_line_range

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1801_09803_gb300 as m
    m.build.build()
    m.lib()
    return m


def test_grid_shards_through_the_library(xc):
    L = xs.gen_lines(43, 0, 200_000, 990.0, 1075.0)
    E, g = xs.gen_states(43, 1000)
    o = np.argsort(L["nu"], kind="stable")
    S = {k: v[o] for k, v in L.items()}
    base = xs.conditions_for(xs.WORKLOADS["C3"])
    conds = [xc.make_condition(base[i]["T"], base[i]["P"]) for i in range(0, 32, 2)]   # 16 conditions
    nu_A, step, n, cut = 1000.0, 1.0 / 128.0, 8193, 5.0
    world = 4
    results = {}
    for prec in ("fp64", "fp32"):
        opts = xc.make_opts("voigt_w4", prec, cut)
        with xc.Engine(0) as eng:
            eng.load_lines(S, assume_sorted=True)
            eng.set_states(E, g)
            full = eng.cross_section_batched(conds, xc.make_grid(nu_A, step, n), opts)
        parts, halo = [], []
        for r in range(world):
            k0, k1 = grid_shard(n, world, r)
            l0, l1 = halo_line_range(S["nu"], nu_A, step, k0, k1, cut)
            halo.append(l1 - l0)
            with xc.Engine(0) as eng:
                eng.load_lines({k: v[l0:l1] for k, v in S.items()}, assume_sorted=True)
                eng.set_states(E, g)
                parts.append(eng.cross_section_batched(conds, xc.make_grid(nu_A + k0 * step, step, k1 - k0), opts))
        sharded = np.concatenate(parts, axis=1)
        results[prec] = (full, sharded)
        assert max(halo) < len(S["nu"])   # each shard holds only its halo range
    full64, shard64 = results["fp64"]
    assert np.array_equal(full64, shard64)
    full32, shard32 = results["fp32"]
    m = full32 > 1e-6 * full32.max(axis=1, keepdims=True)
    diff = float(np.max(np.abs(shard32[m] - full32[m]) / full32[m]))
    band = float(np.max(np.abs(shard32.sum(axis=1) - full32.sum(axis=1)) / full32.sum(axis=1)))
    print(f"grid shards through the library: FP64 bit-exact; FP32 max rel {diff:.3g}, band {band:.3g}")
    assert diff < 2e-5 and band < 1e-6
