"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (written here; the FP32 bound is w4 region-boundary jumps plus FP32 rounding):
  FP64 path: max relative error <= 1e-5 over bins above 1e-6 of the peak
             (measured ~1e-12: only the rounding of exp/pow differs).
  FP32 path: max relative error <= 2e-4 over bins above 1e-6 of the peak and
             relative error of the band-integrated cross section <= 1e-5.
Integer / index work (sort, permutation, eval counts) is bit-exact.
"""
import os

import numpy as np
import pytest

import xcsynth as xs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROFILES = ["doppler", "lorentz", "voigt_w4", "voigt_gh_binned", "voigt_gh_sampled", "doppler_binned",
            "lorentz_binned"]
TOL64 = 1e-5
TOL32 = 2e-4
TOL32_BAND = 1e-5
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1801_09803_gb300 as m
    m.build.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def eng(xc):
    e = xc.Engine(0)
    yield e
    e.close()


def metrics(got, ref, frac=1e-6):
    got = np.asarray(got)
    ref = np.asarray(ref)
    if ref.max() <= 0:
        return float(np.max(np.abs(got))), 0.0
    m = ref > frac * ref.max()
    mr = float(np.max(np.abs(got[m] - ref[m]) / ref[m]))
    band = float(abs(got.sum() - ref.sum()) / ref.sum())
    return mr, band


def oracle_sigma(oracle, lines, E, g, T, P, nu_A, step, n, profile, cut, wm=0.0, n_gh=20, quantity="absorption",
                 threshold=None, **kw):
    Q, dQ = oracle.partition_function(E, g, T)
    c = oracle.make_condition(T, P, Q, dQ, **kw)
    return oracle.cross_section(lines, c, nu_A, step, n,
                                oracle.make_opts(profile, cut, wm, n_gh, quantity=quantity, threshold=threshold),
                                nthreads=NTHREADS)


# ------------------------------------------------------------------ sort
def test_sort_is_stable_and_exact(eng, xc):
    L = xs.gen_lines(101, 0, 100_003, 1000.0, 1100.0)
    L["nu"][5000:5100] = L["nu"][77]          # ties: equal wavenumbers keep input order
    L["nu"][9000] = L["nu"][9001]
    eng.load_lines(L)
    got = eng.get_lines()
    perm = eng.get_permutation()
    order = np.argsort(L["nu"], kind="stable")
    assert np.array_equal(perm, order.astype(np.uint32))
    for k in L:
        assert np.array_equal(got[k], L[k][order]), k


def test_sort_device_input_and_many_tiles(eng, xc):
    L = xs.gen_lines(102, 0, 2_000_000, 0.0, 10000.0)
    eng.load_lines({k: torch.as_tensor(v).cuda() for k, v in L.items()})
    order = np.argsort(L["nu"], kind="stable")
    assert np.array_equal(eng.get_permutation(), order.astype(np.uint32))
    assert np.array_equal(eng.get_lines()["nu"], L["nu"][order])


def test_assume_sorted_and_invalid_input(eng, xc):
    L = xs.gen_lines(103, 0, 5000, 1000.0, 1010.0)
    o = np.argsort(L["nu"], kind="stable")
    S = {k: v[o] for k, v in L.items()}
    eng.load_lines(S, assume_sorted=True)
    assert np.array_equal(eng.get_permutation(), np.arange(5000, dtype=np.uint32))
    with pytest.raises(xc.XcError) as ei:
        eng.load_lines(L, assume_sorted=True)
    assert ei.value.status == 1
    for field, bad in (("nu", 0.0), ("nu", np.nan), ("A", -1.0), ("gamma_ref", -0.1), ("elower", np.inf)):
        B = {k: v.copy() for k, v in L.items()}
        B[field][17] = bad
        with pytest.raises(xc.XcError) as ei:
            eng.load_lines(B)
        assert ei.value.status == 1, field


# ------------------------------------------------------------------ Q(T), line parameters, counts
def test_partition_function(xc, oracle_lib):
    E, g = xs.gen_states(7, 5000)
    T = np.array([300.0, 296.0, 1000.0, 3000.0, 12345.0])
    Q, dQ = xc.partition_function(E, g, T)
    for i, t in enumerate(T):
        q, dq = oracle_lib.partition_function(E, g, t)
        assert abs(Q[i] - q) <= 1e-13 * q
        assert abs(dQ[i] - dq) <= 1e-12 * dq
    Td = torch.as_tensor(T).cuda()
    Qd, _ = xc.partition_function(torch.as_tensor(E).cuda(), torch.as_tensor(g).cuda(), Td)
    assert np.allclose(Qd.cpu().numpy(), Q, rtol=1e-15, atol=0)


def test_line_params(eng, xc, oracle_lib):
    L = xs.gen_lines(104, 0, 20000, 0.0, 10000.0)
    E, g = xs.gen_states(104, 3000)
    eng.load_lines(L)
    eng.set_states(E, g)
    S = eng.get_lines()
    for T, P in ((300.0, 1e-3), (1500.0, 1.0), (3000.0, 10.0)):
        I, a, gm = eng.line_params(xc.make_condition(T, P, gamma_scale=1.05, n_shift=0.1))
        Q, dQ = oracle_lib.partition_function(E, g, T)
        c = oracle_lib.make_condition(T, P, Q, dQ, gamma_scale=1.05, n_shift=0.1)
        for l in range(0, 20000, 397):
            assert I[l] == pytest.approx(oracle_lib.intensity(S["nu"][l], S["elower"][l], S["A"][l], S["g_up"][l], c),
                                         rel=1e-13, abs=0)
            assert a[l] == pytest.approx(oracle_lib.alpha_doppler(S["nu"][l], c), rel=1e-14, abs=0)
            assert gm[l] == pytest.approx(oracle_lib.gamma_lorentz(S["gamma_ref"][l], S["n_T"][l], c), rel=1e-13, abs=0)


@pytest.mark.parametrize("wm", [0.0, 500.0, 20.0])
def test_count_evals_exact(eng, xc, oracle_lib, wm):
    L = xs.gen_lines(105, 0, 30000, 0.0, 60.0)
    E, g = xs.gen_states(105, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(0.0, 0.01, 6001)
    conds = [xc.make_condition(T, P) for T, P in ((400.0, 0.1), (1500.0, 1.0))]
    got = eng.count_evals(conds, grid, xc.make_opts("voigt_w4", "fp64", 25.0, wm))
    exp = 0
    for cd in conds:
        Q, dQ = oracle_lib.partition_function(E, g, cd.T)
        exp += oracle_lib.count_evals(L, oracle_lib.make_condition(cd.T, cd.P, Q, dQ), 0.0, 0.01, 6001,
                                      oracle_lib.make_opts("voigt_w4", 25.0, wm))
    assert got == exp


# ------------------------------------------------------------------ cross sections
def _small_case():
    # 8000 lines over 80 cm-1, grid of 3001 points (ragged last window), cut 3 cm-1,
    # lines on both sides of the grid edges
    L = xs.gen_lines(106, 0, 8000, 995.0, 1035.0)
    E, g = xs.gen_states(106, 2000)
    return L, E, g, 1000.0, 0.01, 3001


@pytest.mark.parametrize("profile", PROFILES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cross_section_profiles(eng, xc, oracle_lib, profile, precision):
    L, E, g, nu_A, step, n = _small_case()
    eng.load_lines(L)
    eng.set_states(E, g)
    T, P = 1200.0, 0.5
    got = eng.cross_section(xc.make_condition(T, P), xc.make_grid(nu_A, step, n),
                            xc.make_opts(profile, precision, 3.0, n_gh=20))
    ref = oracle_sigma(oracle_lib, L, E, g, T, P, nu_A, step, n, profile, 3.0)
    mr, band = metrics(got, ref)
    print(f"{profile} {precision}: max rel {mr:.3g}, band {band:.3g}")
    if precision == "fp64":
        assert mr < TOL64 and band < TOL64
    else:
        assert mr < TOL32 and band < TOL32_BAND


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_conditions(eng, xc, oracle_lib, precision):
    # the 8 x 4 (T, P) sweep of the batched workload on a small line list, cut 25
    L = xs.gen_lines(107, 0, 20000, 0.0, 200.0)
    E, g = xs.gen_states(107, 5000)
    eng.load_lines(L)
    eng.set_states(E, g)
    W = xs.WORKLOADS["C3"]
    conds = xs.conditions_for(W)
    nu_A, step, n = 0.0, 0.01, 20001
    sel = list(range(32)) if precision == "fp32" else [0, 13, 31]
    cx = [xc.make_condition(conds[i]["T"], conds[i]["P"]) for i in sel]
    got = eng.cross_section_batched(cx, xc.make_grid(nu_A, step, n), xc.make_opts("voigt_w4", precision, 25.0))
    worst = (0.0, 0.0)
    for j, i in enumerate(sel):
        if precision == "fp32" and i % 5 != 0:
            continue  # oracle on a subset of the conditions keeps the test short
        ref = oracle_sigma(oracle_lib, L, E, g, conds[i]["T"], conds[i]["P"], nu_A, step, n, "voigt_w4", 25.0)
        mr, band = metrics(got[j], ref)
        worst = (max(worst[0], mr), max(worst[1], band))
    print(f"batched {precision}: worst max rel {worst[0]:.3g}, band {worst[1]:.3g}")
    tol = (TOL64, TOL64) if precision == "fp64" else (TOL32, TOL32_BAND)
    assert worst[0] < tol[0] and worst[1] < tol[1]


def test_tensor_core_partition_on_offset_grid(eng, xc, oracle_lib):
    """The integer far tests, block ranges and line records on a grid that starts
    between line positions and has a step that is not a power of ten (the far/near/
    centre-zone partition must still count every pair once), 24 conditions, and the
    per-kernel statistics of the timed sweep."""
    L = xs.gen_lines(112, 0, 15000, 900.0, 1100.0)
    E, g = xs.gen_states(112, 3000)
    eng.load_lines(L)
    eng.set_states(E, g)
    base = xs.conditions_for(xs.WORKLOADS["C3"])
    conds = [base[i] for i in range(0, 32) if i % 4 != 3]        # 24 conditions, P <= 1 bar
    cx = [xc.make_condition(c["T"], c["P"]) for c in conds]
    nu_A, step, n = 912.3456, 0.0137, 12345
    grid = xc.make_grid(nu_A, step, n)
    eng.set_timing(True)
    try:
        tc = eng.cross_section_batched(cx, grid, xc.make_opts("voigt_w4", "fp32", 10.0))
        far_ms, main_ms, cz_ms, mma = eng.sweep_kernels()
        cu = eng.cross_section_batched(cx, grid, xc.make_opts("voigt_w4", "fp32", 10.0, tensor_cores=False))
        far2, main2, cz2, mma2 = eng.sweep_kernels()
    finally:
        eng.set_timing(False)
    assert mma > 0 and far_ms > 0 and main_ms > 0 and cz_ms > 0
    assert mma2 == 0 and far2 < 0 and main2 > 0
    # the far-wing kernel's evaluations (its own test, counted separately): part of the
    # algorithmic count, and none without the tensor cores
    o = xc.make_opts("voigt_w4", "fp32", 10.0)
    total = eng.count_evals(cx, grid, o)
    n_far = eng.count_far_evals(cx, grid, o)
    print(f"far-wing evaluations {n_far} of {total} ({n_far / total:.3f})")
    assert 0 < n_far <= total
    assert eng.count_far_evals(cx, grid, xc.make_opts("voigt_w4", "fp32", 10.0, tensor_cores=False)) == 0
    m = cu > 1e-6 * cu.max(axis=1, keepdims=True)
    diff = float(np.max(np.abs(tc[m] - cu[m]) / cu[m]))
    full = np.where(m, np.abs(tc - cu) / np.where(m, cu, 1.0), 0.0)
    ci, ki = np.unravel_index(np.argmax(full), full.shape)
    worst, worst_cu = 0.0, 0.0
    for i in (0, 11, 23, int(ci)):
        ref = oracle_sigma(oracle_lib, L, E, g, conds[i]["T"], conds[i]["P"], nu_A, step, n, "voigt_w4", 10.0)
        worst = max(worst, metrics(tc[i], ref)[0])
        worst_cu = max(worst_cu, metrics(cu[i], ref)[0])
    print(f"offset grid: tensor-core vs CUDA-core {diff:.3g} (condition {ci}, point {ki}, "
          f"{tc[ci, ki]:.6g} vs {cu[ci, ki]:.6g}; {int((full > 2e-5).sum())} points), vs oracle: tensor-core "
          f"{worst:.3g}, CUDA-core {worst_cu:.3g}; {mma} MMAs")
    assert diff < 2e-5 and worst < TOL32


@pytest.mark.parametrize("n_cond", [16, 20, 33])
def test_batched_tensor_core_far_wings(eng, xc, oracle_lib, n_cond):
    """FP32 Voigt w4 with >= 16 conditions sums the far wings on the tensor cores
    (ragged last 128-point block, padded condition groups); the result must match
    the oracle like the CUDA-core path does, and the two FP32 paths each other."""
    L = xs.gen_lines(110, 0, 20000, 0.0, 200.0)
    E, g = xs.gen_states(110, 5000)
    eng.load_lines(L)
    eng.set_states(E, g)
    W = xs.WORKLOADS["C3"]
    base = xs.conditions_for(W)
    conds = [base[i % 32] for i in range(n_cond)]
    cx = [xc.make_condition(c["T"], c["P"]) for c in conds]
    nu_A, step, n = 0.0, 0.01, 20001
    grid = xc.make_grid(nu_A, step, n)
    tc = eng.cross_section_batched(cx, grid, xc.make_opts("voigt_w4", "fp32", 25.0))
    cu = eng.cross_section_batched(cx, grid, xc.make_opts("voigt_w4", "fp32", 25.0, tensor_cores=False))
    worst = (0.0, 0.0)
    worst_cu = 0.0
    for i in range(n_cond):
        ref = oracle_sigma(oracle_lib, L, E, g, conds[i]["T"], conds[i]["P"], nu_A, step, n, "voigt_w4", 25.0)
        mr, band = metrics(tc[i], ref)
        mr2, _ = metrics(cu[i], ref)
        if max(mr, mr2) > 2e-5:
            print(f"  condition {i}: tensor-core path {mr:.3g}, CUDA-core path {mr2:.3g}")
        worst = (max(worst[0], mr), max(worst[1], band))
        worst_cu = max(worst_cu, mr2)
    print(f"  CUDA-core path, all conditions: {worst_cu:.3g}; tuning: {eng.tuning()}")
    m = cu > 1e-6 * cu.max(axis=1, keepdims=True)
    rel = (tc[m] - cu[m]) / cu[m]
    diff = float(np.max(np.abs(rel)))
    full = np.where(m, np.abs(tc - cu) / np.where(m, cu, 1.0), 0.0)
    ci, ki = np.unravel_index(np.argmax(full), full.shape)
    print(f"  largest tensor/CUDA-core difference at condition {ci}, point {ki} (block {ki // 128}, "
          f"offset {ki % 128}): {tc[ci, ki]:.6g} vs {cu[ci, ki]:.6g}")
    print(f"tensor-core far wings, {n_cond} conditions: vs oracle {worst[0]:.3g} band {worst[1]:.3g}; "
          f"vs CUDA-core path max {diff:.3g}, mean {float(np.mean(rel)):.3g}")
    assert worst[0] < TOL32 and worst[1] < TOL32_BAND
    assert diff < 2e-5
    assert np.all(tc >= 0)


W4_SHAPES = [(4, 16), (2, 32), (4, 8), (8, 8), (8, 4), (8, 2), (8, 1)]


def test_every_w4_tile_shape(eng, xc, oracle_lib):
    """Every compiled FP32 Voigt w4 tile shape, 33 conditions (padded groups), on the
    CUDA cores and, for the 128-point spans (R = 4), with the tensor-core far wings."""
    L = xs.gen_lines(111, 0, 12000, 0.0, 120.0)
    E, g = xs.gen_states(111, 3000)
    eng.load_lines(L)
    eng.set_states(E, g)
    base = xs.conditions_for(xs.WORKLOADS["C3"])
    conds = [base[i % 32] for i in range(33)]
    cx = [xc.make_condition(c["T"], c["P"]) for c in conds]
    nu_A, step, n = 0.0, 0.01, 12001
    grid = xc.make_grid(nu_A, step, n)
    refs = [oracle_sigma(oracle_lib, L, E, g, c["T"], c["P"], nu_A, step, n, "voigt_w4", 25.0) for c in conds]
    bad = []
    try:
        for R, CG in W4_SHAPES:
            for tcores in ((False, True) if R == 4 else (False,)):
                eng.set_tile_shape(R, CG)
                got = eng.cross_section_batched(cx, grid, xc.make_opts("voigt_w4", "fp32", 25.0, tensor_cores=tcores))
                w = max(metrics(got[i], refs[i]) for i in range(33))
                print(f"R={R} CG={CG} tensor cores {tcores}: max rel {w[0]:.3g}, band {w[1]:.3g}")
                if not (w[0] < TOL32 and w[1] < TOL32_BAND):
                    bad.append((R, CG, tcores, w))
    finally:
        eng.set_tile_shape(0, 0)
    assert not bad, bad


@pytest.mark.parametrize("n_cond", [5, 6, 7, 9])
def test_every_profile_at_odd_condition_counts(eng, xc, oracle_lib, n_cond):
    """Condition counts between the kernel's group sizes (1, 4, 8, 16) run for every profile."""
    L = xs.gen_lines(110, 0, 3000, 1000.0, 1030.0)
    E, g = xs.gen_states(110, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    nu_A, step, n, cut = 995.0, 0.01, 4001, 4.0
    TP = [(300.0 * 1.4 ** i, 0.05 * 2.0 ** i) for i in range(n_cond)]
    grid = xc.make_grid(nu_A, step, n)
    for profile in PROFILES:
        got = eng.cross_section_batched([xc.make_condition(T, P) for T, P in TP], grid,
                                        xc.make_opts(profile, "fp32", cut, n_gh=10))
        for j in (0, n_cond - 1):
            ref = oracle_sigma(oracle_lib, L, E, g, TP[j][0], TP[j][1], nu_A, step, n, profile, cut, n_gh=10)
            mr, band = metrics(got[j], ref)
            assert mr < TOL32 and band < TOL32_BAND, (profile, n_cond, j, mr, band)


@pytest.mark.parametrize("profile", ["voigt_w4", "voigt_gh_binned"])
def test_width_limited_cut(eng, xc, oracle_lib, profile):
    L = xs.gen_lines(108, 0, 10000, 0.0, 100.0)
    E, g = xs.gen_states(108, 2000)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(0.0, 0.01, 10001)
    ref = oracle_sigma(oracle_lib, L, E, g, 1500.0, 1.0, 0.0, 0.01, 10001, profile, 25.0, wm=500.0)
    for precision, tol in (("fp64", (TOL64, TOL64)), ("fp32", (TOL32, TOL32_BAND))):
        got = eng.cross_section(xc.make_condition(1500.0, 1.0), grid, xc.make_opts(profile, precision, 25.0, 500.0))
        mr, band = metrics(got, ref)
        print(f"width-limited {profile} {precision}: {mr:.3g} {band:.3g}")
        assert mr < tol[0] and band < tol[1]
    # the batched FP32 form with per-kernel timing on: its per-condition sweeps run on the
    # stream directly (not captured in a graph), where the timing events are plain records
    eng.set_timing(True)
    try:
        got = eng.cross_section_batched([xc.make_condition(1500.0, 1.0)], grid,
                                        xc.make_opts(profile, "fp32", 25.0, 500.0))
    finally:
        eng.set_timing(False)
    mr, band = metrics(got[0], ref)
    assert mr < TOL32 and band < TOL32_BAND, (mr, band)


@pytest.mark.parametrize("profile", ["doppler_binned", "lorentz_binned"])
def test_binned_profiles_on_a_coarse_grid(eng, xc, oracle_lib, profile):
    """Binned Gaussian / Lorentzian (Eqs. eqn:sig_ij, eqn:sig_lor-2) on a grid up to 50 times
    coarser than the lines, several conditions in one batched sweep, a ragged last tile;
    the FP64 path keeps the area: h sum_k sigma_k = sum_l I_l (to the cut's truncation)."""
    L = xs.gen_lines(109, 0, 30000, 1000.0, 1400.0)
    E, g = xs.gen_states(109, 2000)
    eng.load_lines(L)
    eng.set_states(E, g)
    nu_A, step, n, cut = 990.0, 0.1, 4237, 6.0
    TP = [(300.0, 0.01), (900.0, 0.3), (2000.0, 1.0), (3000.0, 5.0), (1200.0, 0.1), (600.0, 2.0)]
    grid = xc.make_grid(nu_A, step, n)
    got32 = eng.cross_section_batched([xc.make_condition(T, P) for T, P in TP], grid,
                                      xc.make_opts(profile, "fp32", cut))
    worst = (0.0, 0.0)
    for j, (T, P) in enumerate(TP):
        ref = oracle_sigma(oracle_lib, L, E, g, T, P, nu_A, step, n, profile, cut)
        mr, band = metrics(got32[j], ref)
        worst = (max(worst[0], mr), max(worst[1], band))
        if j < 2:
            got64 = eng.cross_section(xc.make_condition(T, P), grid, xc.make_opts(profile, "fp64", cut))
            m64, b64 = metrics(got64, ref)
            assert m64 < TOL64 and b64 < TOL64, (T, P, m64, b64)
            if profile == "doppler_binned":
                Q, _ = oracle_lib.partition_function(E, g, T)
                c = oracle_lib.make_condition(T, P, Q)
                I = sum(oracle_lib.intensity(float(L["nu"][l]), float(L["elower"][l]), float(L["A"][l]),
                                             float(L["g_up"][l]), c) for l in range(len(L["nu"])))
                assert float(np.sum(got64)) * step == pytest.approx(I, rel=1e-9, abs=0)
    print(f"binned {profile} fp32 (6 conditions): worst max rel {worst[0]:.3g}, band {worst[1]:.3g}")
    assert worst[0] < TOL32 and worst[1] < TOL32_BAND


def _strengths(oracle_lib, L, E, g, TP, quantity):
    f = oracle_lib.emissivity if quantity == "emission" else oracle_lib.intensity
    out = np.empty((len(TP), len(L["nu"])))
    for j, (T, P) in enumerate(TP):
        Q, _ = oracle_lib.partition_function(E, g, T)
        c = oracle_lib.make_condition(T, P, Q)
        out[j] = [f(L["nu"][l], L["elower"][l], L["A"][l], L["g_up"][l], c) for l in range(len(L["nu"]))]
    return out


@pytest.mark.parametrize("quantity", ["absorption", "emission"])
def test_emission_and_intensity_thresholds(eng, xc, oracle_lib, quantity):
    """Eq. (e:emiss) and the constant / HITRAN intensity thresholds, FP64 and the FP32 batched
    sweep (18 conditions: far wings on the tensor cores).  Threshold values sit where no
    (line, condition) strength is within 1e-6 of them, so the FP64 keep decisions are unique."""
    L = xs.gen_lines(111, 0, 3000, 1000.0, 1040.0)
    E, g = xs.gen_states(111, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    nu_A, step, n, cut = 995.0, 0.01, 5001, 5.0
    TP = [(300.0 * 1.15 ** i, 0.02 * 1.5 ** i) for i in range(18)]
    grid = xc.make_grid(nu_A, step, n)
    S = _strengths(oracle_lib, L, E, g, TP, quantity)
    # constant threshold: a value inside a gap of the sorted strengths near the median
    srt = np.sort(S.ravel())
    mid = len(srt) // 2
    gaps = srt[mid - 500:mid + 500]
    i = int(np.argmax(gaps[1:] / gaps[:-1]))
    I_cut = float(np.sqrt(gaps[i] * gaps[i + 1]))
    # HITRAN threshold: I_crit scaled so that it also sits away from every ratio S / (thr / I_crit)
    o1 = oracle_lib.make_opts(threshold=("hitran", 1020.0, 1.0))
    base = np.array([[oracle_lib.threshold(L["nu"][l], T, o1) for l in range(len(L["nu"]))] for T, _ in TP])
    r = np.sort((S / base).ravel())
    rm = r[len(r) // 2 - 500:len(r) // 2 + 500]
    k = int(np.argmax(rm[1:] / rm[:-1]))
    I_crit = float(np.sqrt(rm[k] * rm[k + 1]))
    for thr in (None, ("constant", I_cut), ("hitran", 1020.0, I_crit)):
        sel = [0, 7, 17]
        refs = {j: oracle_sigma(oracle_lib, L, E, g, TP[j][0], TP[j][1], nu_A, step, n, "voigt_w4", cut,
                                quantity=quantity, threshold=thr) for j in sel}
        if thr is not None:
            kept = S >= (I_cut if thr[0] == "constant" else I_crit * base)
            assert 0.2 < kept.mean() < 0.8
        for j in sel[:2]:
            got = eng.cross_section(xc.make_condition(*TP[j]), grid,
                                    xc.make_opts("voigt_w4", "fp64", cut, quantity=quantity, threshold=thr))
            m64, b64 = metrics(got, refs[j])
            assert m64 < TOL64 and b64 < TOL64, (thr, j, m64, b64)
        conds = [xc.make_condition(T, P) for T, P in TP]
        eng.set_timing(True)
        try:
            got = eng.cross_section_batched(conds, grid, xc.make_opts("voigt_w4", "fp32", cut, quantity=quantity,
                                                                      threshold=thr))
            assert eng.sweep_kernels()[3] > 0   # the tensor-core kernel took the far wings
        finally:
            eng.set_timing(False)
        cu = eng.cross_section_batched(conds, grid, xc.make_opts("voigt_w4", "fp32", cut, tensor_cores=False,
                                                                 quantity=quantity, threshold=thr))
        worst = (0.0, 0.0)
        for j in sel:
            mr, band = metrics(got[j], refs[j])
            worst = (max(worst[0], mr), max(worst[1], band))
            mc, _ = metrics(got[j], cu[j])
            assert mc < 2e-5, (thr, j, mc)
        print(f"{quantity} threshold {thr}: fp32 batched worst max rel {worst[0]:.3g}, band {worst[1]:.3g}")
        assert worst[0] < TOL32 and worst[1] < TOL32_BAND, (thr, worst)


def test_broadener_mixture(eng, xc, oracle_lib):
    """.broad a0 and a1 broadeners mixed 0.6 / 0.4 (Secs. "Broadening parameters", "Mixtures of
    broadeners"): FP64 and the FP32 batched sweep (18 conditions, far wings on the tensor
    cores), a width-limited cut, and the way back to the lines' own widths."""
    L = xs.gen_lines(112, 0, 3000, 1000.0, 1040.0)
    E, g = xs.gen_states(112, 1000)
    j_up = (L["g_up"].astype(np.int32) - 1) // 2
    eng.load_lines(L)
    eng.set_states(E, g)
    a0 = {j: (0.09 - 0.0011 * j, 0.75 - 0.004 * j) for j in range(0, 60, 2)}
    a1 = {(j, j + 1): (0.05 + 0.0007 * j, 0.6) for j in range(0, 60, 3)}
    a1.update({(j, j - 1): (0.04, 0.45 + 0.002 * j) for j in range(1, 60, 4)})
    ob = [oracle_lib.make_broadener("a0", 0.6, 0.07, 0.5, a0), oracle_lib.make_broadener("a1", 0.4, 0.03, 0.7, a1)]
    eng.set_broadening([xc.make_broadener("a0", 0.6, 0.07, 0.5, a0), xc.make_broadener("a1", 0.4, 0.03, 0.7, a1)],
                       j_up=j_up)
    nu_A, step, n, cut = 995.0, 0.01, 5001, 5.0
    TP = [(300.0 * 1.15 ** i, 0.02 * 1.5 ** i) for i in range(18)]
    grid = xc.make_grid(nu_A, step, n)

    def ref(j, o):
        Q, dQ = oracle_lib.partition_function(E, g, TP[j][0])
        c = oracle_lib.make_condition(TP[j][0], TP[j][1], Q, dQ)
        return oracle_lib.cross_section_broad(L, j_up, ob, c, nu_A, step, n, o, nthreads=NTHREADS)

    sel = [0, 9, 17]
    refs = {j: ref(j, oracle_lib.make_opts("voigt_w4", cut)) for j in sel}
    for j in sel[:2]:
        got = eng.cross_section(xc.make_condition(*TP[j]), grid, xc.make_opts("voigt_w4", "fp64", cut))
        m64, b64 = metrics(got, refs[j])
        assert m64 < TOL64 and b64 < TOL64, (j, m64, b64)
    conds = [xc.make_condition(T, P) for T, P in TP]
    eng.set_timing(True)
    try:
        got = eng.cross_section_batched(conds, grid, xc.make_opts("voigt_w4", "fp32", cut))
        assert eng.sweep_kernels()[3] > 0
    finally:
        eng.set_timing(False)
    cu = eng.cross_section_batched(conds, grid, xc.make_opts("voigt_w4", "fp32", cut, tensor_cores=False))
    worst = (0.0, 0.0)
    for j in sel:
        mr, band = metrics(got[j], refs[j])
        worst = (max(worst[0], mr), max(worst[1], band))
        assert metrics(got[j], cu[j])[0] < 2e-5
    print(f"broadener mixture fp32 batched: worst max rel {worst[0]:.3g}, band {worst[1]:.3g}")
    assert worst[0] < TOL32 and worst[1] < TOL32_BAND
    # width-limited cut uses the mixture widths too
    r = ref(5, oracle_lib.make_opts("voigt_w4", 25.0, 200.0))
    for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
        got = eng.cross_section(conds[5], grid, xc.make_opts("voigt_w4", prec, 25.0, 200.0))
        assert metrics(got, r)[0] < tol, prec
    # under a mixture the adjoint has no per-line gradients of the line list's widths (EINVAL);
    # an empty mixture returns to the lines' own widths
    with pytest.raises(xc.XcError):
        eng.cross_section_vjp(conds[:1], grid, xc.make_opts("voigt_w4", "fp64", cut), np.ones((1, n)), per_line=True)
    eng.set_broadening([])
    plain = eng.cross_section(conds[0], grid, xc.make_opts("voigt_w4", "fp64", cut))
    r0 = oracle_sigma(oracle_lib, L, E, g, TP[0][0], TP[0][1], nu_A, step, n, "voigt_w4", cut)
    assert metrics(plain, r0)[0] < TOL64


@pytest.mark.parametrize("beta,norm", [(False, False), (True, False), (False, True), (True, True)])
def test_vectorized_voigt(eng, xc, oracle_lib, beta, norm):
    """Eq. (e:fast-v) with beta = 1 or Eq. (e:beta), and VVN: FP64 and the FP32 batched sweep
    (6 conditions) against the oracle; the exact zone 1.5 cm^-1, so the reference wing
    carries most points."""
    L = xs.gen_lines(113, 0, 2000, 3000.0, 3040.0)
    E, g = xs.gen_states(113, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    nu_A, step, n, cut, split = 2990.0, 0.05, 1301, 8.0, 1.5
    TP = [(2500.0, 0.3), (800.0, 1.0), (1500.0, 0.05), (3000.0, 3.0), (400.0, 0.5), (2000.0, 0.01)]
    grid = xc.make_grid(nu_A, step, n)
    kw = dict(vv_split=split, vv_beta=beta, vv_norm=norm)

    def ref(j):
        Q, dQ = oracle_lib.partition_function(E, g, TP[j][0])
        c = oracle_lib.make_condition(TP[j][0], TP[j][1], Q, dQ)
        return oracle_lib.cross_section(L, c, nu_A, step, n, oracle_lib.make_opts("voigt_vv", cut, **kw),
                                        nthreads=NTHREADS)

    refs = {j: ref(j) for j in (0, 3, 5)}
    for j in (0, 3):
        got = eng.cross_section(xc.make_condition(*TP[j]), grid, xc.make_opts("voigt_vv", "fp64", cut, **kw))
        m64, b64 = metrics(got, refs[j])
        assert m64 < TOL64 and b64 < TOL64, (j, m64, b64)
    got = eng.cross_section_batched([xc.make_condition(T, P) for T, P in TP], grid,
                                    xc.make_opts("voigt_vv", "fp32", cut, **kw))
    worst = (0.0, 0.0)
    for j, r in refs.items():
        mr, band = metrics(got[j], r)
        worst = (max(worst[0], mr), max(worst[1], band))
    print(f"vectorized voigt beta={beta} norm={norm}: fp32 worst max rel {worst[0]:.3g}, band {worst[1]:.3g}")
    assert worst[0] < TOL32 and worst[1] < TOL32_BAND


def test_vectorized_voigt_reference_wing_outside_region_one(eng, xc, oracle_lib):
    """The FP32 kernel evaluates the reference wing as a region-I rational in u only when
    a_ref (split + g) >= 15 in grid steps (a_ref = sqrt(ln 2) h / (alpha / nu), about 3e4
    here); a split far below the grid step and a Lorentz width near zero (P = 1e-4 bar) take
    the other branch (the w4 Voigt in x, y) for every line.  Against the oracle, FP32.
    With the exact zone far below a grid step the band is carried by the one or two grid
    points a few 1e-4 steps from a line centre, where the reference Voigt has |x| + y < 15
    and the complex w4 is evaluated in FP32 (8e-5 relative at the one such point of this
    list); so the band is held to the pointwise bound here, not to the band bound."""
    L = xs.gen_lines(114, 0, 1000, 3000.0, 3020.0)
    E, g = xs.gen_states(114, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    nu_A, step, n, cut = 2995.0, 0.05, 601, 5.0
    TP = [(300.0, 1e-4), (1500.0, 1e-4), (3000.0, 2e-4)]
    kw = dict(vv_split=1e-5, vv_beta=True, vv_norm=False)
    grid = xc.make_grid(nu_A, step, n)
    got = eng.cross_section_batched([xc.make_condition(T, P) for T, P in TP], grid,
                                    xc.make_opts("voigt_vv", "fp32", cut, **kw))
    for j, (T, P) in enumerate(TP):
        Q, dQ = oracle_lib.partition_function(E, g, T)
        c = oracle_lib.make_condition(T, P, Q, dQ)
        ref = oracle_lib.cross_section(L, c, nu_A, step, n, oracle_lib.make_opts("voigt_vv", cut, **kw),
                                       nthreads=NTHREADS)
        mr, band = metrics(got[j], ref)
        assert mr < TOL32 and band < TOL32, (j, mr, band)


def test_c1_full_size(eng, xc, oracle_lib):
    """The single-condition FP64 workload at full size: 1e5 lines, 200001 points."""
    W = xs.WORKLOADS["C1"]
    L = xs.gen_lines(W.seed, 0, W.n_lines, W.nu_lo, W.nu_hi)
    E, g = xs.gen_states(W.seed, W.n_states)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
    ref = oracle_sigma(oracle_lib, L, E, g, 1000.0, 1.0, W.grid_lo, W.step, W.n_points, "voigt_w4", 25.0)
    for precision in ("fp64", "fp32"):
        got = eng.cross_section(xc.make_condition(1000.0, 1.0), grid, xc.make_opts("voigt_w4", precision, 25.0))
        mr, band = metrics(got, ref)
        print(f"C1 {precision}: max rel {mr:.3g}, band {band:.3g}")
        if precision == "fp64":
            assert mr < TOL64 and band < TOL64
        else:
            assert mr < TOL32 and band < TOL32_BAND


def test_edge_cases(eng, xc, oracle_lib):
    E, g = xs.gen_states(109, 500)
    eng.set_states(E, g)
    opts64 = xc.make_opts("voigt_w4", "fp64", 1.0)
    opts32 = xc.make_opts("voigt_w4", "fp32", 1.0)
    # lines entirely outside the grid and beyond the cut: exact zeros
    L = xs.gen_lines(109, 0, 100, 2000.0, 2001.0)
    eng.load_lines(L)
    for o in (opts64, opts32):
        s = eng.cross_section(xc.make_condition(800.0, 1.0), xc.make_grid(1000.0, 0.01, 1001), o)
        assert np.all(s == 0.0)
    # one grid point; empty grid
    L = xs.gen_lines(110, 0, 300, 999.5, 1000.5)
    eng.load_lines(L)
    ref = oracle_sigma(oracle_lib, L, E, g, 800.0, 1.0, 1000.0, 0.01, 1, "voigt_w4", 1.0)
    for o, tol in ((opts64, TOL64), (opts32, TOL32)):
        s = eng.cross_section(xc.make_condition(800.0, 1.0), xc.make_grid(1000.0, 0.01, 1), o)
        assert abs(s[0] - ref[0]) <= tol * ref[0]
        z = eng.cross_section_batched([xc.make_condition(800.0, 1.0)], xc.make_grid(1000.0, 0.01, 0), o)
        assert z.shape == (1, 0)
    # empty line list
    eng.load_lines({k: v[:0] for k, v in L.items()})
    for o in (opts64, opts32):
        s = eng.cross_section(xc.make_condition(800.0, 1.0), xc.make_grid(1000.0, 0.01, 301), o)
        assert np.all(s == 0.0)
    # invalid arguments are rejected
    eng.load_lines(L)
    with pytest.raises(xc.XcError):
        eng.cross_section(xc.make_condition(-5.0, 1.0), xc.make_grid(1000.0, 0.01, 10), opts64)
    with pytest.raises(xc.XcError):
        eng.cross_section(xc.make_condition(500.0, 1.0), xc.make_grid(1000.0, -0.01, 10), opts64)
    with pytest.raises(xc.XcError):
        eng.cross_section(xc.make_condition(500.0, 1.0), xc.make_grid(1000.0, 0.01, 10),
                          xc.make_opts("voigt_gh_binned", "fp32", 1.0, n_gh=0))


def test_option_errors(eng, xc):
    """Bad option values are EINVAL; the paths that do not implement an option refuse it
    with EUNSUPPORTED (the adjoint, the allocation-free entry point); reloading the lines
    drops a broadener mixture."""
    import ctypes as C
    L = xs.gen_lines(114, 0, 500, 1000.0, 1005.0)
    E, g = xs.gen_states(114, 500)
    eng.load_lines(L)
    eng.set_states(E, g)
    cond, grid = xc.make_condition(900.0, 1.0), xc.make_grid(999.0, 0.01, 701)

    def status(fn):
        try:
            fn()
        except xc.XcError as e:
            return e.status
        return 0

    bad = []
    o = xc.make_opts("voigt_vv", "fp64", 3.0); o.vv_split = -1.0; bad.append(o)
    o = xc.make_opts("voigt_vv", "fp64", 3.0); o.vv_flags = 4; bad.append(o)
    o = xc.make_opts("voigt_w4", "fp64", 3.0); o.quantity = 2; bad.append(o)
    o = xc.make_opts("voigt_w4", "fp64", 3.0); o.threshold = 3; bad.append(o)
    bad.append(xc.make_opts("voigt_w4", "fp64", 3.0, threshold=("hitran", 0.0, 1e-29)))
    bad.append(xc.make_opts("voigt_w4", "fp64", 3.0, threshold=("constant", -1.0)))
    o = xc.make_opts("voigt_w4", "fp64", 3.0); o.profile = 8; bad.append(o)
    for o in bad:
        assert status(lambda: eng.cross_section(cond, grid, o)) in (1, 5), (o.profile, o.quantity, o.threshold)
    # broadening misuse
    a1 = xc.make_broadener("a1", 1.0, 0.05, 0.5, {(3, 4): (0.06, 0.6)})
    assert status(lambda: eng.set_broadening([a1])) == 1                      # a1 needs J'
    dup = xc.make_broadener("a0", 1.0, 0.05, 0.5, {2: (0.06, 0.6), 3: (0.07, 0.6)})
    dup._keep[0][:] = 2                                                       # two rows keyed J'' = 2
    assert status(lambda: eng.set_broadening([dup])) == 1
    neg = xc.make_broadener("constant", -0.5, 0.05, 0.5)
    assert status(lambda: eng.set_broadening([neg])) == 1
    many = [xc.make_broadener("constant", 0.1, 0.05, 0.5)] * 9
    assert status(lambda: eng.set_broadening(many)) == 1
    # the adjoint refuses emission, thresholds and the Vectorized Voigt
    gs = np.ones((1, grid.n))
    for o in (xc.make_opts("voigt_w4", "fp64", 3.0, quantity="emission"),
              xc.make_opts("voigt_w4", "fp64", 3.0, threshold=("constant", 1e-30)),
              xc.make_opts("voigt_vv", "fp64", 3.0)):
        assert status(lambda: eng.cross_section_vjp([cond], grid, o, gs)) == 5
    # the allocation-free entry point refuses them too (and the binned profiles)
    o_ = np.argsort(L["nu"], kind="stable")
    dl = {k: torch.from_numpy(v[o_]).cuda() for k, v in L.items()}
    dE, dg = torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda()
    out = torch.zeros((1, grid.n), dtype=torch.float64, device="cuda:0")
    Ls = xc.XcLines(dl["nu"].data_ptr(), dl["elower"].data_ptr(), dl["A"].data_ptr(), dl["gamma_ref"].data_ptr(),
                    dl["n_T"].data_ptr(), dl["g_up"].data_ptr(), dl["j_lo"].data_ptr(), xc.XC_MEM_DEVICE)
    arr = (xc.XcCondition * 1)(cond)
    for o in (xc.make_opts("voigt_w4", "fp32", 3.0, quantity="emission"),
              xc.make_opts("voigt_w4", "fp32", 3.0, threshold=("hitran", 2000.0, 1e-29)),
              xc.make_opts("voigt_vv", "fp32", 3.0), xc.make_opts("doppler_binned", "fp32", 3.0)):
        rc = xc.lib().xc_cross_section_batched_static(C.byref(Ls), len(o_), dE.data_ptr(), dg.data_ptr(), len(E),
                                                      arr, 1, C.byref(grid), C.byref(o), out.data_ptr(), None)
        assert rc == 5, (o.profile, rc)
    # a mixture belongs to the lines it was set for
    plain = eng.cross_section(cond, grid, xc.make_opts("voigt_w4", "fp64", 3.0))
    eng.set_broadening([xc.make_broadener("constant", 1.0, 0.2, 0.5)])
    wide = eng.cross_section(cond, grid, xc.make_opts("voigt_w4", "fp64", 3.0))
    assert not np.allclose(wide, plain, rtol=1e-3, atol=0)
    eng.load_lines(L)
    again = eng.cross_section(cond, grid, xc.make_opts("voigt_w4", "fp64", 3.0))
    assert np.array_equal(again, plain)


def test_deterministic_and_memory_kinds_agree(eng, xc):
    L = xs.gen_lines(111, 0, 20000, 0.0, 100.0)
    E, g = xs.gen_states(111, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(0.0, 0.01, 10001)
    conds = [xc.make_condition(T, 1.0) for T in (300.0, 900.0, 2700.0)]
    o = xc.make_opts("voigt_w4", "fp32", 25.0)
    a = eng.cross_section_batched(conds, grid, o)
    b = eng.cross_section_batched(conds, grid, o)
    d = torch.zeros((3, 10001), dtype=torch.float64, device="cuda:0")
    eng.cross_section_batched(conds, grid, o, d)
    assert np.array_equal(a, b)
    assert np.array_equal(a, d.cpu().numpy())
