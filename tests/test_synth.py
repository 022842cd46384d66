"""The seeded input generator: determinism, slice invariance and the stated recipe."""
import numpy as np

import xcsynth as xs


def test_slice_invariance_and_determinism():
    a = xs.gen_lines(7, 0, 5000, 1000.0, 3000.0)
    b = xs.gen_lines(7, 1234, 1000, 1000.0, 3000.0, chunk=97)
    for k in a:
        assert np.array_equal(a[k][1234:2234], b[k]), k
    c = xs.gen_lines_at(7, np.array([1234, 4000, 17]), 1000.0, 3000.0)
    for k in a:
        assert np.array_equal(c[k], a[k][[1234, 4000, 17]]), k
    d = xs.gen_lines(8, 0, 5000, 1000.0, 3000.0)
    assert not np.array_equal(a["nu"], d["nu"])


def test_splitmix_reference_values():
    # SplitMix64 output function on counter 0 with seed 0 is 0 (fixed point of the mixer),
    # and the first mix of the golden-ratio increment is the well-known first SplitMix64 output.
    z = xs._mix(np.array([0], np.uint64))
    assert int(z[0]) == 0
    z = xs._mix(np.array([0x9E3779B97F4A7C15], np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_recipe_ranges():
    n = 200_000
    L = xs.gen_lines(11, 0, n, 0.0, 10000.0)
    assert L["nu"].min() > 0.0 and L["nu"].max() <= 10000.0
    assert L["elower"].min() >= 0.0 and L["elower"].max() <= 20000.0
    # exponential with scale 3000: mean of the unclamped part ~ 3000 (clamp is rare: e^-6.7)
    assert abs(L["elower"].mean() - 3000.0) < 40.0
    assert L["j_lo"].min() == 0 and L["j_lo"].max() == 50
    ju = (L["g_up"].astype(int) - 1) // 2
    dj = ju - L["j_lo"]
    assert set(np.unique(dj)) <= {-1, 0, 1}
    assert np.all(ju >= 0)
    la = np.log10(L["A"].astype(np.float64))
    assert la.min() >= -6.0 - 1e-6 and la.max() <= 2.0 + 1e-6
    assert abs(la.mean() + 2.0) < 0.05
    assert L["gamma_ref"].min() >= 0.02 - 1e-7 and L["gamma_ref"].max() <= 0.1 + 1e-7
    assert L["n_T"].min() >= 0.4 - 1e-7 and L["n_T"].max() <= 0.8 + 1e-7
    # nu uniform: each of 10 bands holds ~10 %
    h, _ = np.histogram(L["nu"], bins=10, range=(0, 10000))
    assert np.all(np.abs(h / n - 0.1) < 0.005)


def test_states():
    E, g = xs.gen_states(3, 5000)
    assert E.shape == (5000,) and g.dtype == np.int32
    assert np.all(g % 2 == 1) and g.min() >= 1 and g.max() <= 101
    E2, g2 = xs.gen_states(3, 5000)
    assert np.array_equal(E, E2) and np.array_equal(g, g2)


def test_workloads():
    assert xs.WORKLOADS["C1"].n_points == 200001
    assert xs.WORKLOADS["C2"].n_points == 1000001
    assert xs.WORKLOADS["C5"].n_points == 2000001
    c3 = xs.WORKLOADS["C3"]
    assert c3.n_conditions == 32
    T = np.array(c3.temperatures)
    assert abs(T[0] - 300.0) < 1e-9 and abs(T[-1] - 3000.0) < 1e-9
    assert np.allclose(np.diff(np.log(T)), np.log(10) / 7)


def test_torch_generator_matches_numpy():
    torch = __import__("pytest").importorskip("torch")
    a = xs.gen_lines(77, 1000, 20000, 0.0, 20000.0)
    b = xs.gen_lines_torch(77, 1000, 20000, 0.0, 20000.0, device="cpu", chunk=7001)
    for k in ("nu", "j_lo", "g_up", "gamma_ref", "n_T"):
        assert np.array_equal(a[k], b[k].numpy()), k
    for k in ("elower", "A"):  # library log1p / pow may differ in the last bit before rounding
        d = np.abs(a[k].astype(np.float64) - b[k].numpy().astype(np.float64)) / np.maximum(np.abs(a[k]), 1e-30)
        assert d.max() <= 1.2e-7, k
