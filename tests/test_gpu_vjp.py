"""Adjoint (VJP) of the cross section on the GPU, through the C ABI.

Checked against (a) the FP64 oracle's analytic gradient on the same lines and
(b) central finite differences (h = 1e-4 relative) of the GPU FP64 forward,
for the retrieval-style loss L = sum (sigma - sigma_target)^2 with the target
from T x 1.03 and gamma_ref x 1.05 (gamma_scale = 1.05).
Tolerance: 1e-4 relative (FP64 adjoint: 1e-8 against the oracle).
"""
import os

import numpy as np
import pytest

import xcsynth as xs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
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


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("profile", ["voigt_w4", "doppler", "lorentz", "voigt_gh_binned"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vjp_matches_oracle_gradient(eng, xc, oracle_lib, profile, precision):
    L = xs.gen_lines(201, 0, 3000, 1000.0, 1020.0)
    E, g = xs.gen_states(201, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    S = eng.get_lines()                       # sorted order, as the library reports per-line grads
    nu_A, step, n, cut = 995.0, 0.01, 3001, 2.0
    TP = [(800.0, 0.1), (1600.0, 1.0), (1600.0, 0.1)]
    rng = np.random.default_rng(5)
    # FP64: random-sign weights (heavy cancellation, exact comparison).  FP32: positive
    # weights, so the comparison measures the kernel's rounding rather than the
    # condition number of a cancelling sum (the finite-difference test below uses the
    # real, mixed-sign loss gradient).
    gs = rng.standard_normal((len(TP), n)) if precision == "fp64" else 0.5 + rng.random((len(TP), n))
    conds = [xc.make_condition(T, P, gamma_scale=1.05, n_shift=0.02) for T, P in TP]
    r = eng.cross_section_vjp(conds, xc.make_grid(nu_A, step, n), xc.make_opts(profile, precision, cut), gs)
    oc = []
    for T, P in TP:
        Q, dQ = oracle_lib.partition_function(E, g, T)
        oc.append(oracle_lib.make_condition(T, P, Q, dQ, gamma_scale=1.05, n_shift=0.02))
    ref = oracle_lib.cross_section_vjp(S, oc, nu_A, step, n, oracle_lib.make_opts(profile, cut), gs)
    tol = 1e-8 if precision == "fp64" else 1e-4
    errs = {"dT": _rel(r["dT"], ref["dT"])}
    if profile != "doppler":
        errs.update(dP=_rel(r["dP"], ref["dP"]), ds=_rel(r["d_gamma_scale"], [ref["d_gamma_scale"]]),
                    dn=_rel(r["d_n_shift"], [ref["d_n_shift"]]))
        for key in ("d_gamma_ref_line", "d_n_line"):
            # element by element, on every line whose gradient is not negligible
            big = np.abs(ref[key]) > 1e-3 * np.abs(ref[key]).max()
            assert big.sum() >= 10, key
            errs[key] = _rel(r[key][big], ref[key][big])
    else:
        assert np.all(r["dP"] == 0.0) and r["d_gamma_scale"][0] == 0.0
    print(profile, precision, {k: f"{v:.2g}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < tol, (k, v)


W_LINES_C4 = xs.WORKLOADS["C4"].n_lines


@pytest.mark.parametrize("profile", ["voigt_w4", "lorentz", "doppler", "voigt_gh_binned"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vjp_broadener_mixture_matches_oracle(eng, xc, oracle_lib, profile, precision):
    """The adjoint under a mixture of .broad broadeners (an a0 table, an a1 table and a
    constant; Secs. "Broadening parameters", "Mixtures of broadeners"): dT, dP, the global
    scalars and the per-broadener gradients (a factor on each broadener's gamma_0 values,
    a shift of its n values) against the oracle's, and the same scalars through the
    plain entry point.  Positive weights for FP32 as in the test above.  Tolerance
    1e-8 (FP64) and 1e-4 (FP32) relative."""
    L = xs.gen_lines(205, 0, 2000, 1000.0, 1015.0)
    E, g = xs.gen_states(205, 1000)
    j_up = (L["g_up"].astype(np.int32) - 1) // 2
    eng.load_lines(L)
    eng.set_states(E, g)
    S = eng.get_lines()
    perm = eng.get_permutation()
    a0 = {j: (0.09 - 0.0011 * j, 0.75 - 0.004 * j) for j in range(0, 60, 2)}
    a1 = {(j, j + 1): (0.05 + 0.0007 * j, 0.6) for j in range(0, 60, 3)}
    spec = [("a0", 0.5, 0.07, 0.5, a0), ("a1", 0.3, 0.03, 0.7, a1), ("constant", 0.2, 0.04, 0.65, None)]
    eng.set_broadening([xc.make_broadener(*sp) for sp in spec], j_up=j_up)
    ob = [oracle_lib.make_broadener(*sp) for sp in spec]
    nu_A, step, n, cut = 995.0, 0.01, 2501, 2.0
    TP = [(800.0, 0.1), (1600.0, 1.0), (2400.0, 0.3)]
    rng = np.random.default_rng(7)
    gs = rng.standard_normal((len(TP), n)) if precision == "fp64" else 0.5 + rng.random((len(TP), n))
    conds = [xc.make_condition(T, P, gamma_scale=1.0, n_shift=0.01) for T, P in TP]
    opts = xc.make_opts(profile, precision, cut)
    try:
        r = eng.cross_section_vjp_broadening(conds, xc.make_grid(nu_A, step, n), opts, gs, len(spec))
        r2 = eng.cross_section_vjp(conds, xc.make_grid(nu_A, step, n), opts, gs, per_line=False)
    finally:
        eng.set_broadening([])
    oc = []
    for T, P in TP:
        Q, dQ = oracle_lib.partition_function(E, g, T)
        oc.append(oracle_lib.make_condition(T, P, Q, dQ, gamma_scale=1.0, n_shift=0.01))
    ref = oracle_lib.cross_section_vjp_broad(S, j_up[perm], ob, oc, nu_A, step, n, oracle_lib.make_opts(profile, cut),
                                             gs)
    tol = 1e-8 if precision == "fp64" else 1e-4
    errs = {"dT": _rel(r["dT"], ref["dT"])}
    if profile != "doppler":
        errs.update(dP=_rel(r["dP"], ref["dP"]), ds=_rel(r["d_gamma_scale"], [ref["d_gamma_scale"]]),
                    dn=_rel(r["d_n_shift"], [ref["d_n_shift"]]),
                    dg0=_rel(r["d_gamma0_broad"], ref["d_gamma0_broad"]),
                    dnb=_rel(r["d_n_broad"], ref["d_n_broad"]))
        errs["plain entry"] = max(_rel(r2["dT"], r["dT"]), _rel(r2["dP"], r["dP"]),
                                  _rel(r2["d_gamma_scale"], r["d_gamma_scale"]))
    print("mixture", profile, precision, {k: f"{v:.2g}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < tol, (k, v)


def _c4_problem(xc, eng, n_lines, seed_off=0):
    W = xs.WORKLOADS["C4"]
    L = xs.gen_lines(W.seed + seed_off, 0, n_lines, W.nu_lo, W.nu_hi)
    E, g = xs.gen_states(W.seed, W.n_states)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
    TP = [(T, P) for T in W.temperatures for P in W.pressures]
    return W, L, E, g, grid, TP


def test_vjp_c4_against_central_differences(eng, xc):
    """Differentiation workload (C1 generator and grid, 2 x 2 conditions) on 2e5 lines."""
    W, L, E, g, grid, TP = _c4_problem(xc, eng, 200_000)
    o64 = xc.make_opts("voigt_w4", "fp64", 25.0)
    o32 = xc.make_opts("voigt_w4", "fp32", 25.0)
    dev = "cuda:0"
    # target: T x 1.03, gamma_ref x 1.05 (through gamma_scale)
    tgt = torch.zeros((len(TP), grid.n), dtype=torch.float64, device=dev)
    eng.cross_section_batched([xc.make_condition(T * 1.03, P, gamma_scale=1.05) for T, P in TP], grid, o64, tgt)

    def loss(Ts, Ps, s=1.0, dn=0.0):
        out = torch.zeros((len(TP), grid.n), dtype=torch.float64, device=dev)
        eng.cross_section_batched([xc.make_condition(T, P, gamma_scale=s, n_shift=dn) for T, P in zip(Ts, Ps)],
                                  grid, o64, out)
        return float(((out - tgt) ** 2).sum()), out

    T0 = [T for T, _ in TP]
    P0 = [P for _, P in TP]
    L0, s0 = loss(T0, P0)
    gsig = 2.0 * (s0 - tgt)
    conds = [xc.make_condition(T, P) for T, P in TP]
    r64 = eng.cross_section_vjp(conds, grid, o64, gsig, per_line=False)
    r32 = eng.cross_section_vjp(conds, grid, o32, gsig, per_line=False)
    h = 1e-4
    for c in range(len(TP)):
        Tp, Tm = list(T0), list(T0)
        Tp[c] *= 1 + h
        Tm[c] *= 1 - h
        fd = (loss(Tp, P0)[0] - loss(Tm, P0)[0]) / (2 * h * T0[c])
        Pp, Pm = list(P0), list(P0)
        Pp[c] *= 1 + h
        Pm[c] *= 1 - h
        fdp = (loss(T0, Pp)[0] - loss(T0, Pm)[0]) / (2 * h * P0[c])
        for r in (r64, r32):
            assert float(r["dT"][c]) == pytest.approx(fd, rel=1e-4, abs=0), (c, float(r["dT"][c]), fd)
            assert float(r["dP"][c]) == pytest.approx(fdp, rel=1e-4, abs=0), (c, float(r["dP"][c]), fdp)
    fds = (loss(T0, P0, s=1 + h)[0] - loss(T0, P0, s=1 - h)[0]) / (2 * h)
    dn = 1e-4
    fdn = (loss(T0, P0, dn=dn)[0] - loss(T0, P0, dn=-dn)[0]) / (2 * dn)
    for r in (r64, r32):
        assert float(r["d_gamma_scale"][0]) == pytest.approx(fds, rel=1e-4, abs=0)
        assert float(r["d_n_shift"][0]) == pytest.approx(fdn, rel=1e-4, abs=0)


def test_vjp_c4_full_size_against_central_differences(eng, xc):
    """The differentiation workload at its full size: 1e7 lines (C1 generator and grid,
    200001 points, cut 25 cm^-1), T in {800, 1600} K x P in {0.1, 1} bar, the loss
    sum (sigma - sigma_target)^2 with the target from T x 1.03 and gamma_ref x 1.05.
    The FP32 adjoint is compared with central differences (h = 1e-4 relative) of the
    FP64 forward: dL/dT_c and dL/dP_c for the two extreme conditions (only sigma_c
    depends on them, so each difference needs that condition's forward alone), and the
    global dL/d(gamma_scale) and dL/d(n_shift).  Tolerance 1e-4 relative."""
    W, L, E, g, grid, TP = _c4_problem(xc, eng, W_LINES_C4)
    o64 = xc.make_opts("voigt_w4", "fp64", 25.0)
    o32 = xc.make_opts("voigt_w4", "fp32", 25.0)
    dev = "cuda:0"
    nc = len(TP)
    tgt = torch.zeros((nc, grid.n), dtype=torch.float64, device=dev)
    eng.cross_section_batched([xc.make_condition(T * 1.03, P, gamma_scale=1.05) for T, P in TP], grid, o64, tgt)
    s0 = torch.zeros_like(tgt)
    eng.cross_section_batched([xc.make_condition(T, P) for T, P in TP], grid, o64, s0)
    gsig = 2.0 * (s0 - tgt)
    r32 = eng.cross_section_vjp([xc.make_condition(T, P) for T, P in TP], grid, o32, gsig, per_line=False)
    one = torch.zeros((1, grid.n), dtype=torch.float64, device=dev)

    def loss_c(c, T, P, s=1.0, dn=0.0):   # condition c's part of the loss
        eng.cross_section_batched([xc.make_condition(T, P, gamma_scale=s, n_shift=dn)], grid, o64, one)
        return float(((one[0] - tgt[c]) ** 2).sum())

    h = 1e-4
    report = {}
    for c in (0, nc - 1):
        T, P = TP[c]
        fdT = (loss_c(c, T * (1 + h), P) - loss_c(c, T * (1 - h), P)) / (2 * h * T)
        fdP = (loss_c(c, T, P * (1 + h)) - loss_c(c, T, P * (1 - h))) / (2 * h * P)
        report[f"dT{c}"] = (float(r32["dT"][c]), fdT)
        report[f"dP{c}"] = (float(r32["dP"][c]), fdP)
    fds = sum(loss_c(c, T, P, s=1 + h) - loss_c(c, T, P, s=1 - h) for c, (T, P) in enumerate(TP)) / (2 * h)
    fdn = sum(loss_c(c, T, P, dn=h) - loss_c(c, T, P, dn=-h) for c, (T, P) in enumerate(TP)) / (2 * h)
    report["d_gamma_scale"] = (float(r32["d_gamma_scale"][0]), fds)
    report["d_n_shift"] = (float(r32["d_n_shift"][0]), fdn)
    print("C4 full size, FP32 adjoint vs central differences:",
          {k: f"{abs(a - b) / abs(b):.2g}" for k, (a, b) in report.items()})
    for k, (a, b) in report.items():
        assert a == pytest.approx(b, rel=1e-4, abs=0), (k, a, b)


def test_vjp_c4_subset_against_oracle(eng, xc, oracle_lib):
    """CPU FP64 reference gradient on a seeded 1e4-line subset of the C4 list."""
    W = xs.WORKLOADS["C4"]
    idx = xs.subset_indices(W.n_lines, 10_000, 44)
    L = xs.gen_lines_at(W.seed, idx, W.nu_lo, W.nu_hi)
    E, g = xs.gen_states(W.seed, W.n_states)
    eng.load_lines(L)
    eng.set_states(E, g)
    S = eng.get_lines()
    grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
    TP = [(T, P) for T in W.temperatures for P in W.pressures]
    gs = np.random.default_rng(9).standard_normal((len(TP), W.n_points))
    r = eng.cross_section_vjp([xc.make_condition(T, P) for T, P in TP], grid, xc.make_opts("voigt_w4", "fp32", 25.0),
                              gs)
    oc = []
    for T, P in TP:
        Q, dQ = oracle_lib.partition_function(E, g, T)
        oc.append(oracle_lib.make_condition(T, P, Q, dQ))
    ref = oracle_lib.cross_section_vjp(S, oc, W.grid_lo, W.step, W.n_points, oracle_lib.make_opts("voigt_w4", 25.0),
                                       gs)
    assert _rel(r["dT"], ref["dT"]) < 1e-4
    assert _rel(r["dP"], ref["dP"]) < 1e-4
    assert _rel(r["d_gamma_scale"], [ref["d_gamma_scale"]]) < 1e-4
    assert _rel(r["d_n_shift"], [ref["d_n_shift"]]) < 1e-4
    # per-line gradients, element by element on the lines that carry a non-negligible one
    for key in ("d_gamma_ref_line", "d_n_line"):
        big = np.abs(ref[key]) > 1e-3 * np.abs(ref[key]).max()
        assert big.sum() >= 100, key
        assert _rel(r[key][big], ref[key][big]) < 1e-4, key


def test_autograd_function(eng, xc):
    L = xs.gen_lines(203, 0, 5000, 1000.0, 1050.0)
    E, g = xs.gen_states(203, 1000)
    eng.load_lines(L)
    eng.set_states(E, g)
    grid = xc.make_grid(1000.0, 0.01, 5001)
    opts = xc.make_opts("voigt_w4", "fp32", 25.0)
    T = torch.tensor([900.0, 1700.0], dtype=torch.float64, requires_grad=True)
    P = torch.tensor([0.5, 1.0], dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    nsh = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
    sig = xc.cross_section_autograd(eng, T, P, s, nsh, grid, opts)
    w = torch.linspace(-1, 1, grid.n, dtype=torch.float64, device=sig.device)
    (sig * w).sum().backward()
    r = eng.cross_section_vjp([xc.make_condition(900.0, 0.5), xc.make_condition(1700.0, 1.0)], grid, opts,
                              w.expand(2, -1).contiguous(), per_line=False)
    # the gradients are ~1e-23: relative tolerance only (the default absolute one would pass anything)
    assert torch.allclose(T.grad, r["dT"].cpu(), rtol=1e-10, atol=0)
    assert torch.allclose(P.grad, r["dP"].cpu(), rtol=1e-10, atol=0)
    assert float(T.grad.abs().min()) > 0
    assert float(s.grad) == pytest.approx(float(r["d_gamma_scale"][0]), abs=0)
