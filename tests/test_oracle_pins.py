"""Pins of the FP64 oracle against facts outside itself.

Each test checks one part of the oracle against a closed form, a textbook
relation, a library routine computed by a different method, a limit, an
invariant or brute force, so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import scipy.stats as st

import xcsynth as xs

LN2 = math.log(2.0)


# ---------------------------------------------------------------- constants
def test_second_radiation_constant(oracle_lib):
    # CODATA 2018: c2 = hc/k = 1.438776877... cm K
    assert abs(oracle_lib.c2() - 1.438776877) < 1e-9


# ------------------------------------------------------ Q(T), Eq. (e:pf)
def test_partition_two_level_and_limits(oracle_lib):
    c2 = 1.438776877503933802
    E = np.array([0.0, 1234.5])
    g = np.array([3, 7], np.int32)
    for T in (50.0, 296.0, 3000.0):
        Q, dQ = oracle_lib.partition_function(E, g, T)
        x = c2 * 1234.5 / T
        assert Q == pytest.approx(3 + 7 * math.exp(-x), rel=1e-14, abs=0)
        assert dQ == pytest.approx(7 * math.exp(-x) * x / T, rel=1e-13, abs=0)
    # T -> infinity: every state counts fully
    Es, gs = xs.gen_states(5, 5000)
    Q, _ = oracle_lib.partition_function(Es, gs, 1e14)
    assert Q == pytest.approx(gs.sum(), rel=1e-8, abs=0)
    # T -> 0: only the ground level (E = 0) survives
    Q0, _ = oracle_lib.partition_function(E, g, 1.0)
    assert Q0 == pytest.approx(3.0, rel=1e-14, abs=0)


def test_partition_derivative_matches_finite_difference(oracle_lib):
    E, g = xs.gen_states(9, 5000)
    for T in (300.0, 1500.0):
        h = T * 1e-5
        Qp, _ = oracle_lib.partition_function(E, g, T + h)
        Qm, _ = oracle_lib.partition_function(E, g, T - h)
        _, dQ = oracle_lib.partition_function(E, g, T)
        assert dQ == pytest.approx((Qp - Qm) / (2 * h), rel=1e-7, abs=0)


# --------------------------------------------- intensity, Eq. (e:int)
def test_intensity_equals_einstein_population_difference(oracle_lib):
    """Two-level system: integrated absorption = A g_u/(8 pi c nu^2 g_l) (n_l - g_l/g_u n_u)
    with Boltzmann fractions n = g e^{-c2 E/T}/Q (the Einstein-coefficient relation of
    Hilborn, Am. J. Phys. 50 (1982) 982, written in wavenumber units)."""
    c2 = 1.438776877503933802
    c_cm = 2.99792458e10
    El, nu = 250.0, 1800.0
    gl, gu, A = 5.0, 7.0, 12.5
    for T in (296.0, 1000.0, 3000.0):
        Eu = El + nu
        Q = 2.0 + gl * math.exp(-c2 * El / T) + gu * math.exp(-c2 * Eu / T)  # plus a ground level g=2
        nl = gl * math.exp(-c2 * El / T) / Q
        nu_pop = gu * math.exp(-c2 * Eu / T) / Q
        expect = A * gu / (8 * math.pi * c_cm * nu ** 2 * gl) * (nl - gl / gu * nu_pop)
        cond = oracle_lib.make_condition(T, 1.0, Q)
        assert oracle_lib.intensity(nu, El, A, gu, cond) == pytest.approx(expect, rel=1e-12, abs=0)


def test_intensity_structure(oracle_lib):
    cond = oracle_lib.make_condition(1000.0, 1.0, 345.0)
    base = oracle_lib.intensity(2000.0, 1000.0, 1.0, 3.0, cond)
    assert oracle_lib.intensity(2000.0, 1000.0, 2.0, 3.0, cond) == pytest.approx(2 * base, rel=1e-15, abs=0)
    assert oracle_lib.intensity(2000.0, 1000.0, 1.0, 6.0, cond) == pytest.approx(2 * base, rel=1e-15, abs=0)
    # Boltzmann ratio between lower levels
    r = oracle_lib.intensity(2000.0, 3000.0, 1.0, 3.0, cond) / base
    assert r == pytest.approx(math.exp(-1.438776877503934 * 2000.0 / 1000.0), rel=1e-13, abs=0)
    # abundance scales I linearly (Sec. 2.1 remark) and Q divides it
    c2 = oracle_lib.make_condition(1000.0, 1.0, 690.0, abundance=0.25)
    assert oracle_lib.intensity(2000.0, 1000.0, 1.0, 3.0, c2) == pytest.approx(base / 8, rel=1e-15, abs=0)
    # small c2 nu/T: (1 - e^{-x}) -> x, so I -> g A c2 /(8 pi c nu T Q) ; tests the expm1 branch
    hot = oracle_lib.make_condition(1e6, 1.0, 1.0)
    nu = 1e-3
    expect = 1.0 * 1.438776877503934 / (8 * math.pi * 2.99792458e10 * nu * 1e6)
    assert oracle_lib.intensity(nu, 0.0, 1.0, 1.0, hot) == pytest.approx(expect, rel=1e-8, abs=0)


# --------------------------------------------- emissivity, Eq. (e:emiss); thresholds
def test_emissivity_over_intensity_is_planck(oracle_lib):
    """Kirchhoff's law in LTE: emissivity / absorption intensity of the same line equals the
    Planck function in wavenumber units, B(nu, T) = 2 h c^2 nu^3 / (exp(h c nu / k T) - 1)
    (CGS: erg s^-1 cm^-2 sr^-1 per cm^-1), for any Q, degeneracy, A and lower energy."""
    import scipy.constants as sc
    h, c, k = sc.h * 1e7, sc.c * 100.0, sc.k * 1e7
    for T, nu, El, A, g, Q in ((296.0, 1000.0, 0.0, 1.0, 3.0, 100.0), (1500.0, 3750.5, 2000.0, 25.0, 11.0, 870.0),
                                 (3000.0, 0.37, 15000.0, 1e-5, 1.0, 5000.0), (5000.0, 20000.0, 300.0, 2.0, 7.0, 9e3)):
        cond = oracle_lib.make_condition(T, 1.0, Q)
        B = 2 * h * c ** 2 * nu ** 3 / math.expm1(h * c * nu / (k * T))
        ratio = oracle_lib.emissivity(nu, El, A, g, cond) / oracle_lib.intensity(nu, El, A, g, cond)
        assert ratio == pytest.approx(B, rel=1e-12, abs=0)


def test_emissivity_from_upper_state_population(oracle_lib):
    """Emitted power per molecule and steradian = (fraction of molecules in the upper level)
    x A x photon energy / 4 pi, with the upper level's Boltzmann fraction g' e^{-c2 E'/T}/Q."""
    import scipy.constants as sc
    c2 = sc.h * sc.c * 100.0 / sc.k
    El, nu, gu, A, T, Q = 700.0, 2500.0, 9.0, 40.0, 2200.0, 3100.0
    frac = gu * math.exp(-c2 * (El + nu) / T) / Q
    expect = frac * A * (sc.h * 1e7) * (sc.c * 100.0) * nu / (4 * math.pi)
    eps = oracle_lib.emissivity(nu, El, A, gu, oracle_lib.make_condition(T, 1.0, Q))
    assert eps == pytest.approx(expect, rel=1e-12, abs=0)


def test_hitran_dynamic_threshold(oracle_lib):
    """I_crit above nu_crit; below it, I_crit (nu/nu_crit) tanh(c2 nu/2T), which tends to
    I_crit nu/nu_crit where c2 nu >> T and to I_crit c2 nu^2 / (2 T nu_crit) where c2 nu << T."""
    o = oracle_lib.make_opts(threshold=("hitran", 2000.0, 1e-29))
    assert oracle_lib.threshold(2500.0, 296.0, o) == 1e-29
    assert oracle_lib.threshold(1999.0, 50.0, o) == pytest.approx(1e-29 * 1999.0 / 2000.0, rel=1e-12, abs=0)
    nu, T = 0.01, 3000.0
    c2 = 1.438776877503933802
    assert oracle_lib.threshold(nu, T, o) == pytest.approx(1e-29 * c2 * nu * nu / (2 * T * 2000.0), rel=1e-9, abs=0)
    assert oracle_lib.threshold(500.0, 1000.0, o) < oracle_lib.threshold(1000.0, 1000.0, o) < 1e-29
    assert oracle_lib.threshold(123.0, 1000.0, oracle_lib.make_opts(threshold=("constant", 3e-25))) == 3e-25
    assert oracle_lib.threshold(123.0, 1000.0, oracle_lib.make_opts()) == 0.0


@pytest.mark.parametrize("quantity", ["absorption", "emission"])
def test_threshold_leaves_out_exactly_the_weak_lines(oracle_lib, quantity):
    """A cross section with a threshold equals the cross section of the sub-list of lines whose
    strength (chosen in the test from the pinned intensity / emissivity) is at least the
    threshold at their wavenumber."""
    L = xs.gen_lines(33, 0, 400, 100.0, 3000.0)
    T, Q = 900.0, 300.0
    cond = oracle_lib.make_condition(T, 1.0, Q)
    strength = oracle_lib.emissivity if quantity == "emission" else oracle_lib.intensity
    S = np.array([strength(L["nu"][l], L["elower"][l], L["A"][l], L["g_up"][l], cond) for l in range(400)])
    for thr in (("constant", float(np.median(S))), ("hitran", 2000.0, float(np.quantile(S, 0.3)))):
        o = oracle_lib.make_opts("voigt_w4", 5.0, quantity=quantity, threshold=thr)
        cut = np.array([oracle_lib.threshold(L["nu"][l], T, o) for l in range(400)])
        keep = S >= cut
        assert 50 < keep.sum() < 350
        sub = {k: v[keep] for k, v in L.items()}
        o0 = oracle_lib.make_opts("voigt_w4", 5.0, quantity=quantity)
        a = oracle_lib.cross_section(L, cond, 95.0, 0.05, 58201, o, nthreads=2)
        b = oracle_lib.cross_section(sub, cond, 95.0, 0.05, 58201, o0, nthreads=1)
        assert np.allclose(a, b, rtol=1e-13, atol=0)
    # emission sums emissivities, absorption intensities: their ratio line by line is Planck
    if quantity == "emission":
        one = {k: v[:1] for k, v in L.items()}
        e = oracle_lib.cross_section(one, cond, 95.0, 0.05, 58201, oracle_lib.make_opts("doppler", 5.0, quantity="emission"))
        a = oracle_lib.cross_section(one, cond, 95.0, 0.05, 58201, oracle_lib.make_opts("doppler", 5.0))
        m = a > 0
        assert np.allclose(e[m] / a[m], S[0] / oracle_lib.intensity(L["nu"][0], L["elower"][0], L["A"][0],
                                                                    L["g_up"][0], cond), rtol=1e-13, atol=0)


# --------------------------------------------- Vectorized Voigt, Eqs. (e:fast-v), (e:beta)
def test_vectorized_voigt_zones(oracle_lib):
    """Within `split` of the centre the Voigt of the line itself; beyond it the Voigt of a line at
    1 cm^-1 (Doppler HWHM alpha / nu, the same gamma), both against scipy's Voigt to w4's
    accuracy; with a wide Doppler width the wing visibly differs from the line's own Voigt."""
    LN2S = math.sqrt(2 * LN2)
    nu, a, g = 30000.0, 0.2, 0.01
    for D in (0.0, 0.3, -2.5, 3.99):
        v = oracle_lib.voigt_vv(D, a, g, nu)
        assert v == pytest.approx(sp.voigt_profile(D, a / LN2S, g), rel=1.2e-4, abs=0)
    for D in (4.01, -6.0, 20.0):
        v = oracle_lib.voigt_vv(D, a, g, nu)
        ref = sp.voigt_profile(D, a / nu / LN2S, g)
        assert v == pytest.approx(ref, rel=1.2e-4, abs=0)
        own = sp.voigt_profile(D, a / LN2S, g)
        if abs(D) < 10:
            assert abs(own / ref - 1) > 1e-3    # alpha_ref, not alpha, shapes the wing
    # beta makes the profile continuous at the split point; beta = 1 leaves a jump
    left = oracle_lib.voigt_vv(4.0, a, g, nu, beta=True)
    right = oracle_lib.voigt_vv(4.0 * (1 + 1e-13), a, g, nu, beta=True)
    assert right == pytest.approx(left, rel=1e-9, abs=0)
    assert oracle_lib.voigt_vv(4.0 * (1 + 1e-13), a, g, nu) != pytest.approx(left, rel=1e-4, abs=0)
    # a custom split moves the switch
    assert oracle_lib.voigt_vv(3.0, a, g, nu, split=2.0) == pytest.approx(sp.voigt_profile(3.0, a / nu / LN2S, g),
                                                                           rel=1.2e-4, abs=0)


def test_vvn_conserves_each_line_area(oracle_lib):
    """VVN: h sum_k sigma_k equals the summed intensities for lines whose cut lies inside the
    grid, on fine and coarse grids alike; without normalisation the sampled area differs."""
    L = xs.gen_lines(35, 0, 40, 1000.0, 1010.0)
    cond = oracle_lib.make_condition(1900.0, 1.0, 500.0)
    I = sum(oracle_lib.intensity(L["nu"][l], L["elower"][l], L["A"][l], L["g_up"][l], cond) for l in range(40))
    for h in (0.01, 0.3, 1.0):
        N = int(round(30.0 / h)) + 1
        on = oracle_lib.cross_section(L, cond, 990.0, h, N, oracle_lib.make_opts("voigt_vv", 8.0, vv_norm=True),
                                      nthreads=2)
        assert on.sum() * h == pytest.approx(I, rel=1e-12, abs=0)
        if h == 1.0:
            off = oracle_lib.cross_section(L, cond, 990.0, h, N, oracle_lib.make_opts("voigt_vv", 8.0), nthreads=2)
            assert abs(off.sum() * h / I - 1) > 1e-3


def test_cross_section_bruteforce_vectorized_voigt(oracle_lib):
    L = _tiny_lines(6, seed=5, lo=3000.0, hi=3001.0)
    T, P, Q = 2500.0, 0.3, 900.0
    cond = oracle_lib.make_condition(T, P, Q)
    nu_A, h, N, cut = 2993.5, 0.05, 281, 6.0
    sig = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts("voigt_vv", cut, vv_split=1.5))
    c2, c_cm = 1.438776877503933802, 2.99792458e10
    out = np.zeros(N)
    for k in range(N):
        xk = nu_A + k * h
        for l in range(6):
            nu = float(L["nu"][l]); D = xk - nu
            if abs(D) > cut:
                continue
            I = (float(L["g_up"][l]) * float(L["A"][l]) / (8 * math.pi * c_cm * nu * nu)
                 * math.exp(-c2 * float(L["elower"][l]) / T) * (1 - math.exp(-c2 * nu / T)) / Q)
            al = nu / 2.99792458e8 * math.sqrt(2 * 1.380649e-23 * T * LN2 / (18 * 1.66053906660e-27))
            ga = float(L["gamma_ref"][l]) * (296.0 / T) ** float(L["n_T"][l]) * P
            a_use = al if abs(D) <= 1.5 else al / nu
            out[k] += I * sp.voigt_profile(D, a_use / math.sqrt(2 * LN2), ga)
    m = out > 1e-6 * out.max()
    assert np.max(np.abs(sig[m] - out[m]) / out[m]) < 1.2e-4


# --------------------------------------------- .broad broadening and mixtures
def _read_broad(path):
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        code, g0, n, j = line.split()
        assert code == "a0"
        rows[int(j)] = (float(g0), float(n))
    return rows


def test_broad_a0_table_from_the_paper(oracle_lib):
    """The a0 rows printed for CS in air: at T_ref and P_ref each listed J'' gets its own
    gamma_0; an unlisted J'' the broadener's default; away from T_ref the row's n_L applies."""
    import os
    rows = _read_broad(os.path.join(os.path.dirname(__file__), "golden", "cs_air_a0_broad.txt"))
    assert len(rows) == 7 and rows[3] == (0.0840, 0.089)
    b = oracle_lib.make_broadener("a0", 1.0, 0.07, 0.5, rows)
    ref = oracle_lib.make_condition(296.0, 1.0, 1.0)
    for j, (g0, n) in rows.items():
        assert oracle_lib.gamma_mixture(j, j + 1, [b], ref) == pytest.approx(g0, rel=1e-15, abs=0)
        hot = oracle_lib.make_condition(1184.0, 2.0, 1.0)   # T_ref / T = 1/4
        assert oracle_lib.gamma_mixture(j, j, [b], hot) == pytest.approx(g0 * 0.25 ** n * 2.0, rel=1e-14, abs=0)
    assert oracle_lib.gamma_mixture(10, 11, [b], ref) == pytest.approx(0.07, rel=1e-15, abs=0)


def test_broad_a1_and_mixture_are_weighted_single_broadeners(oracle_lib):
    """a1 keys on (J'', J'); a mixture's HWHM is the rho-weighted sum of each broadener's
    Eq. (e:gamma_L) value (pinned separately), whatever their exponents."""
    a1 = oracle_lib.make_broadener("a1", 0.7, 0.05, 0.6, {(3, 4): (0.08, 0.7), (3, 2): (0.06, 0.4)})
    cst = oracle_lib.make_broadener("constant", 0.3, 0.03, 0.25)
    for T, P in ((296.0, 1.0), (900.0, 0.3), (2500.0, 7.0)):
        c = oracle_lib.make_condition(T, P, 1.0, gamma_scale=1.1, n_shift=0.05)
        for (jl, ju), (g0, n) in (((3, 4), (0.08, 0.7)), ((3, 2), (0.06, 0.4)), ((3, 3), (0.05, 0.6))):
            expect = 0.7 * oracle_lib.gamma_lorentz(g0, n, c) + 0.3 * oracle_lib.gamma_lorentz(0.03, 0.25, c)
            assert oracle_lib.gamma_mixture(jl, ju, [a1, cst], c) == pytest.approx(expect, rel=1e-14, abs=0)
    # two halves of one broadener are that broadener
    half = oracle_lib.make_broadener("constant", 0.5, 0.03, 0.25)
    one = oracle_lib.make_broadener("constant", 1.0, 0.03, 0.25)
    c = oracle_lib.make_condition(700.0, 3.0, 1.0)
    assert oracle_lib.gamma_mixture(0, 1, [half, half], c) == pytest.approx(oracle_lib.gamma_mixture(0, 1, [one], c),
                                                                            rel=1e-15, abs=0)


def test_cross_section_with_a0_broadening_equals_per_line_widths(oracle_lib):
    """One a0 broadener (rho = 1) gives the cross section of the same lines with gamma_ref and
    n_T set to their table rows (values exact in float32)."""
    L = xs.gen_lines(34, 0, 300, 1000.0, 1010.0)
    table = {j: (0.0625 + 0.001953125 * (j % 7), 0.5 + 0.0625 * (j % 3)) for j in range(0, 40, 2)}
    b = oracle_lib.make_broadener("a0", 1.0, 0.046875, 0.75, table)
    j_up = (L["g_up"].astype(np.int32) - 1) // 2
    L2 = dict(L)
    L2["gamma_ref"] = np.array([table.get(int(j), (0.046875, 0.75))[0] for j in L["j_lo"]], np.float32)
    L2["n_T"] = np.array([table.get(int(j), (0.046875, 0.75))[1] for j in L["j_lo"]], np.float32)
    cond = oracle_lib.make_condition(1300.0, 0.8, 400.0)
    o = oracle_lib.make_opts("voigt_w4", 3.0)
    a = oracle_lib.cross_section_broad(L, j_up, [b], cond, 995.0, 0.01, 2001, o, nthreads=2)
    ref = oracle_lib.cross_section(L2, cond, 995.0, 0.01, 2001, o, nthreads=1)
    assert np.allclose(a, ref, rtol=1e-14, atol=0) and ref.max() > 0


@pytest.mark.parametrize("profile", ["voigt_w4", "lorentz", "voigt_gh_binned"])
def test_vjp_with_broadener_mixture_matches_central_differences(oracle_lib, profile):
    """Adjoint under a mixture of broadeners (an a0 table, an a1 table, a constant): dL/dT,
    dL/dP, dL/d(gamma_scale), dL/d(n_shift), and per broadener dL/d(scale of its gamma_0
    values) and dL/d(shift of its n values), each against central differences of the
    forward with that broadener's table rows and defaults perturbed; the per-broadener
    gradients also sum to the global ones (the two identities alone would not catch a
    gradient booked to the wrong broadener)."""
    L = xs.gen_lines(35, 0, 8, 1000.0, 1000.5)
    j_up = (L["g_up"].astype(np.int32) - 1) // 2
    E, gst = xs.gen_states(35, 400)
    nu_A, h, N, cut = 999.0, 0.01, 251, 1.0
    o = oracle_lib.make_opts(profile, cut, n_gh=10)
    gs = np.random.default_rng(1).standard_normal(N)
    a0 = {j: (0.07 - 0.001 * j, 0.7 - 0.01 * j) for j in range(0, 50, 3)}
    a1 = {(int(jl), int(ju)): (0.05 + 0.002 * (k % 5), 0.55 + 0.03 * (k % 4))
          for k, (jl, ju) in enumerate(zip(L["j_lo"][::2], j_up[::2]))}
    spec = [("a0", 0.5, 0.06, 0.6, a0), ("a1", 0.3, 0.04, 0.5, a1), ("constant", 0.2, 0.03, 0.75, None)]

    def mk(i_scale=None, s=1.0, i_shift=None, d=0.0):
        bs = []
        for i, (kind, rho, g0, n, tab) in enumerate(spec):
            f = s if i == i_scale else 1.0
            dn = d if i == i_shift else 0.0
            t2 = None if tab is None else {k: (v[0] * f, v[1] + dn) for k, v in tab.items()}
            bs.append(oracle_lib.make_broadener(kind, rho, g0 * f, n + dn, t2))
        return bs

    T, P = 1100.0, 0.6

    def loss(T=T, P=P, gsc=1.0, nsh=0.0, **kw):
        Q, dQ = oracle_lib.partition_function(E, gst, T)
        c = oracle_lib.make_condition(T, P, Q, dQ, gamma_scale=gsc, n_shift=nsh)
        return float(np.dot(gs, oracle_lib.cross_section_broad(L, j_up, mk(**kw), c, nu_A, h, N, o, nthreads=1)))

    Q, dQ = oracle_lib.partition_function(E, gst, T)
    c = oracle_lib.make_condition(T, P, Q, dQ)
    g = oracle_lib.cross_section_vjp_broad(L, j_up, mk(), [c], nu_A, h, N, o, gs)
    e = 1e-5
    tol = dict(rel=2e-5, abs=0)
    assert g["dT"][0] == pytest.approx((loss(T=T * (1 + e)) - loss(T=T * (1 - e))) / (2 * e * T), **tol)
    assert g["dP"][0] == pytest.approx((loss(P=P * (1 + e)) - loss(P=P * (1 - e))) / (2 * e * P), **tol)
    assert g["d_gamma_scale"] == pytest.approx((loss(gsc=1 + e) - loss(gsc=1 - e)) / (2 * e), **tol)
    assert g["d_n_shift"] == pytest.approx((loss(nsh=e) - loss(nsh=-e)) / (2 * e), **tol)
    for i in range(len(spec)):
        fd_g0 = (loss(i_scale=i, s=1 + e) - loss(i_scale=i, s=1 - e)) / (2 * e)
        fd_n = (loss(i_shift=i, d=e) - loss(i_shift=i, d=-e)) / (2 * e)
        assert g["d_gamma0_broad"][i] == pytest.approx(fd_g0, **tol), (i, g["d_gamma0_broad"][i], fd_g0)
        assert g["d_n_broad"][i] == pytest.approx(fd_n, **tol), (i, g["d_n_broad"][i], fd_n)
        assert abs(g["d_gamma0_broad"][i]) > 1e-3 * abs(g["d_gamma_scale"])   # every broadener matters here
    assert g["d_gamma0_broad"].sum() == pytest.approx(g["d_gamma_scale"], rel=1e-12, abs=0)
    assert g["d_n_broad"].sum() == pytest.approx(g["d_n_shift"], rel=1e-12, abs=0)


# --------------------------------------------- widths, Eqs. (e:alphaD), (e:gamma_L)
def test_doppler_hwhm_textbook_constant(oracle_lib):
    # alpha_D = 3.581e-7 * nu * sqrt(T / M[g/mol])  (the usual practical form)
    for T, nu in ((296.0, 1000.0), (3000.0, 10000.0)):
        cond = oracle_lib.make_condition(T, 1.0, 1.0, mass_da=18.0)
        assert oracle_lib.alpha_doppler(nu, cond) == pytest.approx(3.5812e-7 * nu * math.sqrt(T / 18.0), rel=2e-4, abs=0)
    c1 = oracle_lib.make_condition(400.0, 1.0, 1.0)
    c4 = oracle_lib.make_condition(1600.0, 1.0, 1.0)
    assert oracle_lib.alpha_doppler(2000.0, c4) == pytest.approx(2 * oracle_lib.alpha_doppler(2000.0, c1), rel=1e-15, abs=0)


def test_lorentz_hwhm_scaling(oracle_lib):
    ref = oracle_lib.make_condition(296.0, 1.0, 1.0)
    assert oracle_lib.gamma_lorentz(0.07, 0.5, ref) == pytest.approx(0.07, rel=1e-15, abs=0)
    hot = oracle_lib.make_condition(592.0, 3.0, 1.0)
    assert oracle_lib.gamma_lorentz(0.07, 0.5, hot) == pytest.approx(0.07 * 3.0 / math.sqrt(2.0), rel=1e-14, abs=0)
    sc = oracle_lib.make_condition(592.0, 1.0, 1.0, gamma_scale=1.05, n_shift=0.25)
    assert oracle_lib.gamma_lorentz(0.07, 0.5, sc) == pytest.approx(1.05 * 0.07 * 0.5 ** 0.75, rel=1e-14, abs=0)


# --------------------------------------------- profiles
def test_gauss_is_normal_pdf_with_hwhm(oracle_lib):
    a = 0.037
    sig = a / math.sqrt(2 * LN2)
    for D in (0.0, 0.01, -0.05, 0.2):
        assert oracle_lib.gauss(D, a) == pytest.approx(st.norm.pdf(D, scale=sig), rel=1e-13, abs=0)
    assert oracle_lib.gauss(a, a) == pytest.approx(0.5 * oracle_lib.gauss(0.0, a), rel=1e-14, abs=0)


def test_lorentz_is_cauchy_pdf(oracle_lib):
    g = 0.061
    for D in (0.0, 0.03, -1.0, 24.9):
        assert oracle_lib.lorentz(D, g) == pytest.approx(st.cauchy.pdf(D, scale=g), rel=1e-13, abs=0)


def test_w4_against_faddeeva(oracle_lib):
    """w4's relative accuracy is about 1e-4 (Humlicek 1982); compare with scipy's wofz
    and with mpmath's erfc at 30 digits."""
    xs_ = np.concatenate([np.linspace(-30, 30, 121), [0.0, 0.7071, 3.3, 5.49, 5.51, 14.99, 15.01]])
    ys_ = np.concatenate([np.logspace(-8, 2.3, 40), [0.176, 0.195]])
    worst_abs, worst_re = 0.0, 0.0
    for x in xs_:
        for y in ys_:
            w = oracle_lib.w4(x, y)
            e = sp.wofz(complex(x, y))
            worst_abs = max(worst_abs, abs(w - e) / abs(e))
            worst_re = max(worst_re, abs(w.real - e.real) / abs(e.real))
    # w4 is accurate to ~1e-4 in |w|; Re w alone loses relative accuracy where it is
    # tiny next to Im w (y -> 0 just above s = 5.5, where region II misses exp(-x^2)):
    # measured 3.95e-4 at x = 5.5, y = 1e-8.
    assert worst_abs < 1.2e-4
    assert worst_re < 4.5e-4
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x, y in ((0.3, 0.05), (4.0, 1e-3), (7.0, 0.5), (20.0, 2.0), (2.5, 3.0)):
        z = mp.mpc(x, y)
        e = mp.exp(-z * z) * mp.erfc(-1j * z)
        w = oracle_lib.w4(x, y)
        assert abs(w.real - float(e.real)) / abs(float(e.real)) < 1.2e-4
        assert abs(w.imag - float(e.imag)) / abs(float(e.imag)) < 2e-4


def test_w4_region_boundaries_are_small_jumps(oracle_lib):
    # the four rational forms meet within the approximation's own accuracy
    for x, y in ((15.0 - 0.5 - 1e-9, 0.5), (5.5 - 0.3 - 1e-9, 0.3), (3.0, 0.195 * 3.0 - 0.176 - 1e-9)):
        a = oracle_lib.w4(x, y)
        b = oracle_lib.w4(x + 2e-9, y + (2e-9 if x == 3.0 else 0.0))
        assert abs(a - b) / abs(b) < 2e-4
        assert abs(a.real - b.real) / abs(b.real) < 2e-4


def test_w4_derivative(oracle_lib):
    """F'(t) is the derivative of the same piecewise form (complex finite difference
    inside one region), and approximates the exact w'(z) = -2 z w + 2i/sqrt(pi)."""
    for x, y in ((20.0, 0.5), (7.0, 0.3), (2.0, 1.0), (3.0, 0.05), (0.5, 0.01)):
        w, d = oracle_lib.w4(x, y, deriv=True)
        eps = 1e-6
        fx = (oracle_lib.w4(x + eps, y) - oracle_lib.w4(x - eps, y)) / (2 * eps)
        fy = (oracle_lib.w4(x, y + eps) - oracle_lib.w4(x, y - eps)) / (2 * eps)
        # t = y - i x: dF/dx = -i F'(t), dF/dy = F'(t)
        assert abs(fx - (-1j) * d) < 1e-6 * max(1.0, abs(d))
        assert abs(fy - d) < 1e-6 * max(1.0, abs(d))
        z = complex(x, y)
        exact = -2 * z * sp.wofz(z) + 2j / math.sqrt(math.pi)
        assert abs((-1j) * d - exact) < 5e-3 * abs(exact) + 1e-6


def test_voigt_is_library_voigt_and_limits(oracle_lib):
    a, g = 0.02, 0.03
    sig = a / math.sqrt(2 * LN2)
    for D in (0.0, 0.01, 0.05, -0.3, 5.0, 24.0):
        assert oracle_lib.voigt_w4(D, a, g) == pytest.approx(sp.voigt_profile(D, sig, g), rel=1.2e-4, abs=0)
    # gamma -> 0: Gaussian ; alpha -> 0: Lorentzian (Eqs. e:Gauss, e:lor)
    for D in (0.0, 0.01, 0.03):
        assert oracle_lib.voigt_w4(D, a, 1e-9) == pytest.approx(oracle_lib.gauss(D, a), rel=1.2e-4, abs=0)
    for D in (0.0, 0.01, 0.3):
        assert oracle_lib.voigt_w4(D, 1e-7, g) == pytest.approx(oracle_lib.lorentz(D, g), rel=1.2e-4, abs=0)
    assert oracle_lib.voigt_w4(0.037, a, g) == oracle_lib.voigt_w4(-0.037, a, g)


def test_voigt_unit_area_bruteforce(oracle_lib):
    a, g = 0.02, 0.01
    val, _ = si.quad(lambda D: oracle_lib.voigt_w4(D, a, g), -200, 200, points=[0.0], limit=400)
    assert val == pytest.approx(1.0, abs=2e-4)


def test_gauss_hermite_nodes(oracle_lib):
    for n in (1, 2, 5, 20, 30):
        x, w = oracle_lib.gauss_hermite(n)
        xr, wr = np.polynomial.hermite.hermgauss(n)
        assert np.allclose(x, xr, atol=1e-13, rtol=0)
        assert np.allclose(w, wr, rtol=1e-11, atol=1e-300)
        assert w.sum() == pytest.approx(math.sqrt(math.pi), rel=1e-14, abs=0)
        for k in range(0, 2 * n, 2):  # exact for polynomials of degree <= 2n-1
            assert np.dot(w, x ** k) == pytest.approx(math.gamma(k / 2 + 0.5), rel=1e-10, abs=0)


def test_gh_sampled_voigt_converges_to_voigt(oracle_lib):
    # smooth case (gamma comparable to alpha): 30 nodes match the exact Voigt closely
    a, g = 0.02, 0.03
    sig = a / math.sqrt(2 * LN2)
    for D in (0.0, 0.02, 0.1, 1.0):
        assert oracle_lib.voigt_gh(D, a, g, 30) == pytest.approx(sp.voigt_profile(D, sig, g), rel=2e-3, abs=0)
    val, _ = si.quad(lambda D: oracle_lib.voigt_gh(D, a, g, 20), -np.inf, np.inf, limit=400)
    assert val == pytest.approx(1.0, rel=1e-8, abs=0)


def test_gh_binned_telescopes_and_matches_bin_average(oracle_lib):
    a, g, h = 0.02, 0.015, 0.01
    x, w = oracle_lib.gauss_hermite(20)
    # telescoping over bins k = -K..K: h * sum = pi^-3/2 sum_j w_j [atan(top) - atan(bot)]
    K = 400
    tot = sum(oracle_lib.voigt_gh_binned(k * h, h, a, g, 20) for k in range(-K, K + 1)) * h
    top, bot = (K + 0.5) * h, -(K + 0.5) * h
    expect = sum(w[j] * (math.atan((top - a * x[j] / math.sqrt(LN2)) / g)
                         - math.atan((bot - a * x[j] / math.sqrt(LN2)) / g)) for j in range(20)) / math.pi ** 1.5
    assert tot == pytest.approx(expect, rel=1e-12, abs=0)
    # bin average of the exact Voigt, within the quadrature error of 20 nodes
    sig = a / math.sqrt(2 * LN2)
    for D in (0.0, 0.01, 0.05, 0.5):
        ex, _ = si.quad(lambda u: sp.voigt_profile(u, sig, g), D - h / 2, D + h / 2)
        assert oracle_lib.voigt_gh_binned(D, h, a, g, 20) == pytest.approx(ex / h, rel=5e-3, abs=0)


@pytest.mark.parametrize("h", [0.004, 0.01, 0.1])
def test_binned_gauss_and_lorentz_are_bin_averages(oracle_lib, h):
    """Eqs. (eqn:sig_ij) and (eqn:sig_lor-2): the bin average of the unit-area Gaussian /
    Lorentzian, checked against adaptive quadrature of the library pdfs over the bin."""
    a, g = 0.02, 0.015
    sig = a / math.sqrt(2 * LN2)
    for D in (0.0, 0.3 * h, -0.7 * h, 2.0 * h, 0.05, -0.12, 0.3):
        ex, _ = si.quad(lambda u: st.norm.pdf(u, scale=sig), D - h / 2, D + h / 2, epsabs=0, epsrel=1e-13)
        assert oracle_lib.gauss_binned(D, h, a) == pytest.approx(ex / h, rel=1e-10, abs=0)
        ex, _ = si.quad(lambda u: st.cauchy.pdf(u, scale=g), D - h / 2, D + h / 2, epsabs=0, epsrel=1e-13)
        assert oracle_lib.lorentz_binned(D, h, g) == pytest.approx(ex / h, rel=1e-10, abs=0)
        # symmetric in D
        assert oracle_lib.gauss_binned(-D, h, a) == pytest.approx(oracle_lib.gauss_binned(D, h, a), rel=1e-14, abs=0)
        assert oracle_lib.lorentz_binned(-D, h, g) == pytest.approx(oracle_lib.lorentz_binned(D, h, g), rel=1e-14, abs=0)


def test_binned_gauss_and_lorentz_conserve_area_on_coarse_grids(oracle_lib):
    """The bin averages telescope: h * sum_k equals the profile's integral over the union
    of the bins on any grid, also one far coarser than the line (where sampling fails)."""
    a, g = 0.02, 0.015
    for h in (0.1, 0.037):
        K = 400
        for off in (0.0, 0.013):
            gb = sum(oracle_lib.gauss_binned(k * h + off, h, a) for k in range(-K, K + 1)) * h
            assert gb == pytest.approx(1.0, rel=1e-13, abs=0)
            lb = sum(oracle_lib.lorentz_binned(k * h + off, h, g) for k in range(-K, K + 1)) * h
            top, bot = (K + 0.5) * h + off, -(K + 0.5) * h + off
            assert lb == pytest.approx((st.cauchy.cdf(top, scale=g) - st.cauchy.cdf(bot, scale=g)), rel=1e-12, abs=0)
    # the sampled Gaussian on the coarse grid (points 2.5 alpha either side) keeps ~6 %
    smp = sum(oracle_lib.gauss(k * 0.1 + 0.05, a) for k in range(-40, 41)) * 0.1
    assert smp < 0.1
    # narrow bins: the bin average tends to the sampled profile (error ~ h^2 f''/24)
    for D in (0.0, 0.01, 0.04):
        assert oracle_lib.gauss_binned(D, 1e-5, a) == pytest.approx(oracle_lib.gauss(D, a), rel=1e-7, abs=0)
        assert oracle_lib.lorentz_binned(D, 1e-5, g) == pytest.approx(oracle_lib.lorentz(D, g), rel=1e-7, abs=0)


def test_binned_lorentz_is_one_node_binned_gauss_hermite(oracle_lib):
    """alpha -> 0 collapses Eq. (e:sigma:quad) onto Eq. (eqn:sig_lor-2): every node sits on the
    line centre and the weights sum to sqrt(pi)."""
    g, h = 0.015, 0.01
    for D in (0.0, 0.004, 0.05, 1.3):
        assert oracle_lib.voigt_gh_binned(D, h, 1e-300, g, 20) == pytest.approx(
            oracle_lib.lorentz_binned(D, h, g), rel=1e-13, abs=0)


# --------------------------------------------- full cross sections
def _tiny_lines(n, seed=3, lo=1000.0, hi=1001.0):
    return xs.gen_lines(seed, 0, n, lo, hi)


@pytest.mark.parametrize("profile", ["doppler", "lorentz", "voigt_w4"])
def test_cross_section_bruteforce(oracle_lib, profile):
    L = _tiny_lines(7)
    E, gst = xs.gen_states(3, 500)
    T, P = 1200.0, 0.7
    Q, _ = oracle_lib.partition_function(E, gst, T)
    cond = oracle_lib.make_condition(T, P, Q)
    nu_A, h, N, cut = 999.5, 0.02, 101, 0.6
    sig = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts(profile, cut))
    # independent brute force with library pdfs (scipy), direct per point
    c2, c_cm = 1.438776877503933802, 2.99792458e10
    out = np.zeros(N)
    for k in range(N):
        xk = nu_A + k * h
        for l in range(7):
            nu = float(L["nu"][l]); D = xk - nu
            if abs(D) > cut:
                continue
            I = (float(L["g_up"][l]) * float(L["A"][l]) / (8 * math.pi * c_cm * nu * nu)
                 * math.exp(-c2 * float(L["elower"][l]) / T) * (1 - math.exp(-c2 * nu / T)) / Q)
            al = nu / 2.99792458e8 * math.sqrt(2 * 1.380649e-23 * T * LN2 / (18 * 1.66053906660e-27))
            ga = float(L["gamma_ref"][l]) * (296.0 / T) ** float(L["n_T"][l]) * P
            if profile == "doppler":
                v = st.norm.pdf(D, scale=al / math.sqrt(2 * LN2))
            elif profile == "lorentz":
                v = st.cauchy.pdf(D, scale=ga)
            else:
                v = sp.voigt_profile(D, al / math.sqrt(2 * LN2), ga)
            out[k] += I * v
    tol = 1e-11 if profile != "voigt_w4" else 1.2e-4
    mask = out > 0
    assert np.array_equal(mask, sig > 0)
    assert np.max(np.abs(sig[mask] - out[mask]) / out[mask]) < tol


@pytest.mark.parametrize("profile", ["doppler_binned", "lorentz_binned"])
def test_cross_section_bruteforce_binned(oracle_lib, profile):
    """Sums of bin averages: each (line, bin) by adaptive quadrature of the library pdf."""
    L = _tiny_lines(5, seed=4)
    T, P, Q = 1500.0, 2.0, 700.0
    cond = oracle_lib.make_condition(T, P, Q)
    nu_A, h, N, cut = 999.7, 0.013, 61, 0.35
    sig = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts(profile, cut))
    c2, c_cm = 1.438776877503933802, 2.99792458e10
    out = np.zeros(N)
    for k in range(N):
        xk = nu_A + k * h
        for l in range(5):
            nu = float(L["nu"][l]); D = xk - nu
            if abs(D) > cut:
                continue
            I = (float(L["g_up"][l]) * float(L["A"][l]) / (8 * math.pi * c_cm * nu * nu)
                 * math.exp(-c2 * float(L["elower"][l]) / T) * (1 - math.exp(-c2 * nu / T)) / Q)
            if profile == "doppler_binned":
                al = nu / 2.99792458e8 * math.sqrt(2 * 1.380649e-23 * T * LN2 / (18 * 1.66053906660e-27))
                pdf = lambda u: st.norm.pdf(u, scale=al / math.sqrt(2 * LN2))
            else:
                ga = float(L["gamma_ref"][l]) * (296.0 / T) ** float(L["n_T"][l]) * P
                pdf = lambda u: st.cauchy.pdf(u, scale=ga)
            v, _ = si.quad(pdf, D - h / 2, D + h / 2, epsabs=0, epsrel=1e-12)
            out[k] += I * v / h
    big = out > 1e-9 * out.max()
    assert np.max(np.abs(sig[big] - out[big]) / out[big]) < 1e-9
    assert np.all(np.abs(sig[~big]) <= 2e-9 * out.max())


def test_cutoff_is_inclusive_and_ragged_edges(oracle_lib):
    # a line whose cut lands exactly on grid points (all values exact in binary)
    L = {"nu": np.array([1000.5]), "elower": np.array([0.0], np.float32), "A": np.array([1.0], np.float32),
         "gamma_ref": np.array([0.0625], np.float32), "n_T": np.array([0.5], np.float32),
         "g_up": np.array([1], np.int16), "j_lo": np.array([0], np.int16)}
    cond = oracle_lib.make_condition(296.0, 1.0, 1.0)
    sig = oracle_lib.cross_section(L, cond, 1000.0, 0.125, 9, oracle_lib.make_opts("lorentz", 0.25))
    # points 1000.25 .. 1000.75 (k = 2..6) are within |D| <= 0.25
    assert np.array_equal(np.nonzero(sig)[0], np.arange(2, 7))
    # a line outside the grid still feeds the points within its cut
    L2 = dict(L); L2["nu"] = np.array([999.9])
    sig2 = oracle_lib.cross_section(L2, cond, 1000.0, 0.125, 9, oracle_lib.make_opts("lorentz", 0.25))
    assert np.array_equal(np.nonzero(sig2)[0], np.array([0, 1]))
    # empty line list and an empty grid
    L0 = {k: v[:0] for k, v in L.items()}
    assert np.all(oracle_lib.cross_section(L0, cond, 1000.0, 0.125, 9, oracle_lib.make_opts()) == 0)
    assert oracle_lib.cross_section(L, cond, 1000.0, 0.125, 0, oracle_lib.make_opts()).shape == (0,)


def test_sampled_area_equals_intensity(oracle_lib):
    """Eq. (e:integr): a finely sampled line with a wide cut integrates to I; the truncated
    Lorentzian integrates to I (2/pi) atan(cut/gamma)."""
    L = {"nu": np.array([2000.003]), "elower": np.array([100.0], np.float32), "A": np.array([3.0], np.float32),
         "gamma_ref": np.array([0.05], np.float32), "n_T": np.array([0.6], np.float32),
         "g_up": np.array([5], np.int16), "j_lo": np.array([2], np.int16)}
    cond = oracle_lib.make_condition(1000.0, 1.0, 100.0)
    I = oracle_lib.intensity(2000.003, 100.0, 3.0, 5.0, cond)
    ga = oracle_lib.gamma_lorentz(0.05, 0.6, cond)
    h = 0.001
    nu_A, N = 1990.0, 20001
    s = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts("doppler", 5.0))
    assert s.sum() * h == pytest.approx(I, rel=1e-9, abs=0)
    s = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts("lorentz", 5.0))
    assert s.sum() * h == pytest.approx(I * 2 / math.pi * math.atan(5.0 / ga), rel=1e-6, abs=0)
    s = oracle_lib.cross_section(L, cond, nu_A, h, N, oracle_lib.make_opts("voigt_gh_binned", 5.0))
    # binned GH conserves the area of the truncated profile exactly (telescoping), ~ I atan-limited
    assert s.sum() * h == pytest.approx(I * 2 / math.pi * math.atan(5.0 / ga), rel=2e-5, abs=0)


def test_threads_are_deterministic_and_agree(oracle_lib):
    L = xs.gen_lines(21, 0, 3000, 1000.0, 1010.0)
    cond = oracle_lib.make_condition(800.0, 1.0, 500.0)
    a = oracle_lib.cross_section(L, cond, 995.0, 0.01, 2001, oracle_lib.make_opts("voigt_w4", 3.0), nthreads=1)
    b = oracle_lib.cross_section(L, cond, 995.0, 0.01, 2001, oracle_lib.make_opts("voigt_w4", 3.0), nthreads=4)
    c = oracle_lib.cross_section(L, cond, 995.0, 0.01, 2001, oracle_lib.make_opts("voigt_w4", 3.0), nthreads=4)
    assert np.array_equal(b, c)
    assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_width_limited_cut(oracle_lib):
    L = xs.gen_lines(22, 0, 50, 1000.0, 1002.0)
    cond = oracle_lib.make_condition(1500.0, 1.0, 500.0)
    o = oracle_lib.make_opts("voigt_w4", 25.0, width_mult=10.0)
    n = oracle_lib.count_evals(L, cond, 990.0, 0.01, 2201, o)
    exp_n = 0
    for l in range(50):
        al = oracle_lib.alpha_doppler(L["nu"][l], cond)
        ga = oracle_lib.gamma_lorentz(L["gamma_ref"][l], L["n_T"][l], cond)
        cut = min(25.0, 10.0 * max(al, ga))
        k = np.arange(2201)
        exp_n += int(np.sum(np.abs((990.0 + k * 0.01) - L["nu"][l]) <= cut))
    assert n == exp_n


# --------------------------------------------- adjoint
@pytest.mark.parametrize("profile", ["voigt_w4", "doppler", "lorentz", "voigt_gh_binned", "doppler_binned",
                                     "lorentz_binned"])
def test_vjp_matches_central_differences(oracle_lib, profile):
    L = xs.gen_lines(31, 0, 6, 1000.0, 1000.5)
    E, gst = xs.gen_states(31, 400)
    nu_A, h, N, cut = 999.0, 0.01, 251, 1.0
    o = oracle_lib.make_opts(profile, cut, n_gh=10)
    rng = np.random.default_rng(0)
    gs = rng.standard_normal(N)

    def loss(T, P, s=1.0, dn=0.0, gref=None, nl=None):
        Q, dQ = oracle_lib.partition_function(E, gst, T)
        c = oracle_lib.make_condition(T, P, Q, dQ, gamma_scale=s, n_shift=dn)
        LL = dict(L)
        if gref is not None:
            LL["gamma_ref"] = gref
        if nl is not None:
            LL["n_T"] = nl
        return float(np.dot(gs, oracle_lib.cross_section(LL, c, nu_A, h, N, o)))

    T, P = 900.0, 0.5
    Q, dQ = oracle_lib.partition_function(E, gst, T)
    c = oracle_lib.make_condition(T, P, Q, dQ)
    g = oracle_lib.cross_section_vjp(L, [c], nu_A, h, N, o, gs)
    rel = 1e-5

    def fd(f, x):
        d = x * rel
        return (f(x + d) - f(x - d)) / (2 * d)

    tol = dict(rel=2e-5, abs=1e-30)
    assert g["dT"][0] == pytest.approx(fd(lambda t: loss(t, P), T), **tol)
    assert g["dP"][0] == pytest.approx(fd(lambda p: loss(T, p), P), **tol)
    assert g["d_gamma_scale"] == pytest.approx(fd(lambda s: loss(T, P, s=s), 1.0), **tol)
    d = 1e-5
    fdn = (loss(T, P, dn=d) - loss(T, P, dn=-d)) / (2 * d)
    assert g["d_n_shift"] == pytest.approx(fdn, **tol)
    # per-line gradients, every line: perturb that line's gamma_ref, then its n_T.  Line
    # records are float32, so the perturbed values are exact float32 numbers and the step
    # is their exact difference.  A gradient booked to the wrong line, or with a wrong
    # sign or factor, fails here (the sum identity below would not see a wrong index).
    for field, key in (("gamma_ref", "d_gamma_ref_line"), ("n_T", "d_n_line")):
        base = L[field].copy()
        for l in range(len(base)):
            vp = np.float32(base[l] * (1 + 1e-4))
            vm = np.float32(base[l] * (1 - 1e-4))

            def lg(v):
                a = base.copy()
                a[l] = v
                return loss(T, P, **({"gref": a} if field == "gamma_ref" else {"nl": a}))
            fdl = (lg(vp) - lg(vm)) / (float(vp) - float(vm))
            assert g[key][l] == pytest.approx(fdl, rel=1e-4, abs=0), (field, l, g[key][l], fdl)
    assert g["d_n_line"].sum() == pytest.approx(g["d_n_shift"], rel=1e-12, abs=0)
    # the adjoint covers absorption without a threshold only
    for o2 in (oracle_lib.make_opts(profile, cut, quantity="emission"),
               oracle_lib.make_opts(profile, cut, threshold=("constant", 1e-30))):
        with pytest.raises(RuntimeError):
            oracle_lib.cross_section_vjp(L, [c], nu_A, h, N, o2, gs)


def test_point_evaluation_matches_full_grid(oracle_lib):
    L = xs.gen_lines(23, 0, 3000, 1000.0, 1100.0)
    o = np.argsort(L["nu"], kind="stable")
    S = {k: v[o] for k, v in L.items()}
    E, g = xs.gen_states(23, 500)
    Q, dQ = oracle_lib.partition_function(E, g, 900.0)
    c = oracle_lib.make_condition(900.0, 1.0, Q, dQ)
    for prof, wm in (("voigt_w4", 0.0), ("voigt_gh_binned", 300.0), ("doppler", 0.0)):
        op = oracle_lib.make_opts(prof, 25.0, wm)
        full = oracle_lib.cross_section(S, c, 1000.0, 0.01, 10001, op, nthreads=1)
        ks = np.array([0, 17, 5000, 9999, 10000])
        pts = oracle_lib.cross_section_points(S, c, 1000.0, 0.01, ks, op, nthreads=2)
        assert np.allclose(pts, full[ks], rtol=1e-14, atol=0)
    with pytest.raises(RuntimeError):  # unsorted input is refused
        oracle_lib.cross_section_points(L, c, 1000.0, 0.01, ks, oracle_lib.make_opts(), nthreads=1)
