"""The allocation-free entry point (xc_cross_section_batched_static).

It serves callers that cannot allocate device memory while they run (code in
another framework's memory pool or a fixed memory budget, loops that must not
call cudaMalloc/cudaFree).  It keeps its scratch in a fixed static device array
instead.  These tests call it through the C ABI on device buffers the test owns,
twice in a row for every case (the scratch keeps the previous call's contents,
so the second call checks that everything that must start fresh is cleared),
and compare it with the handle-based xc_cross_section_batched FP32 path within
the FP32 tolerance of the other parity tests; one case is also compared with the
FP64 oracle directly.  The condition counts cover every tile shape the entry
point can pick (groups of 16, 8, 4 and 1 conditions, and the profiles compiled
with fewer group sizes), a condition that brings its own Q(T), and the invalid
inputs it must refuse.  The file is collected last, and passes alone or after
the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import xcsynth as xs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32 = 2e-4


@pytest.fixture(scope="module")
def xc():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1801_09803_gb300 as m
    m.build.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def problem(xc):
    Lh = xs.gen_lines(301, 0, 60000, 0.0, 300.0)
    o = np.argsort(Lh["nu"], kind="stable")
    S = {k: v[o] for k, v in Lh.items()}
    E, g = xs.gen_states(301, 3000)
    return Lh, S, E, g


def _static_call(xc, dl, n, dE, dg, conds, grid, opts, out):
    L = xc.XcLines(dl["nu"].data_ptr(), dl["elower"].data_ptr(), dl["A"].data_ptr(), dl["gamma_ref"].data_ptr(),
                   dl["n_T"].data_ptr(), dl["g_up"].data_ptr(), dl["j_lo"].data_ptr(), xc.XC_MEM_DEVICE)
    arr = (xc.XcCondition * len(conds))(*conds)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return xc.lib().xc_cross_section_batched_static(C.byref(L), n, dE.data_ptr(), dg.data_ptr(), len(dE), arr,
                                                    len(conds), C.byref(grid), C.byref(opts), out.data_ptr(), stream)


def _conds(xc, n_cond):
    """n_cond of the 32 (T, P) conditions of the batched workload, spread over the list."""
    W = xs.WORKLOADS["C3"]
    allc = xs.conditions_for(W)
    return [xc.make_condition(allc[(i * len(allc)) // n_cond]["T"], allc[(i * len(allc)) // n_cond]["P"])
            for i in range(n_cond)]


@pytest.mark.parametrize("n_cond", [1, 3, 5, 12, 32])
@pytest.mark.parametrize("profile", ["voigt_w4", "lorentz", "doppler"])
def test_static_entry_matches_batched(xc, problem, profile, n_cond):
    Lh, S, E, g = problem
    dl = {k: torch.from_numpy(v).cuda() for k, v in S.items()}
    dE, dg = torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda()
    grid = xc.make_grid(0.0, 0.01, 30001)
    conds = _conds(xc, n_cond)
    if n_cond in (3, 12):
        # one condition with its own partition function (Q > 0), here twice what the states
        # give: an entry point that ignored it would be off by a factor of 2
        import oracle
        oracle.build()
        Q, dQ = oracle.partition_function(E, g, conds[0].T)
        conds[0] = xc.make_condition(conds[0].T, conds[0].P, Q=2.0 * Q, dQdT=2.0 * dQ)
    opts = xc.make_opts(profile, "fp32", 25.0)
    with xc.Engine(0) as eng:
        eng.load_lines(Lh)
        eng.set_states(E, g)
        ref = eng.cross_section_batched(conds, grid, opts)
    for attempt in range(2):
        out = torch.full((len(conds), grid.n), float("nan"), dtype=torch.float64, device="cuda:0")
        rc = _static_call(xc, dl, len(S["nu"]), dE, dg, conds, grid, opts, out)
        assert rc == 0, xc.lib().xc_last_error().decode()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        for c in range(len(conds)):
            m = ref[c] > 1e-6 * ref[c].max()
            err = np.max(np.abs(got[c][m] - ref[c][m]) / ref[c][m])
            assert err < TOL32, (profile, n_cond, attempt, c, err)


def test_static_entry_matches_oracle(xc, problem):
    """Directly against the FP64 oracle (not only through the handle path): 3 conditions,
    every grid point above 1e-6 of the peak, the FP32 tolerance of the parity tests."""
    import oracle
    oracle.build()
    Lh, S, E, g = problem
    dl = {k: torch.from_numpy(v).cuda() for k, v in S.items()}
    dE, dg = torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda()
    nu_A, step, n = 0.0, 0.01, 30001
    conds = _conds(xc, 3)
    out = torch.full((len(conds), n), float("nan"), dtype=torch.float64, device="cuda:0")
    rc = _static_call(xc, dl, len(S["nu"]), dE, dg, conds, xc.make_grid(nu_A, step, n),
                      xc.make_opts("voigt_w4", "fp32", 25.0), out)
    assert rc == 0, xc.lib().xc_last_error().decode()
    got = out.cpu().numpy()
    for c, cd in enumerate(conds):
        Q, dQ = oracle.partition_function(E, g, cd.T)
        ref = oracle.cross_section(S, oracle.make_condition(cd.T, cd.P, Q, dQ), nu_A, step, n,
                                   oracle.make_opts("voigt_w4", 25.0), nthreads=16)
        m = ref > 1e-6 * ref.max()
        err = np.max(np.abs(got[c][m] - ref[m]) / ref[m])
        assert err < TOL32, (c, err)


def test_static_entry_rejects_invalid_lines(xc, problem):
    """Unsorted wavenumbers and a negative Einstein A are refused with XC_EINVAL and a
    message that names the fault; the output is left alone."""
    Lh, S, E, g = problem
    dE, dg = torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda()
    grid = xc.make_grid(0.0, 0.01, 30001)
    opts = xc.make_opts("voigt_w4", "fp32", 25.0)
    conds = _conds(xc, 3)
    cases = []
    U = {k: v.copy() for k, v in S.items()}
    U["nu"][5000] = S["nu"][5001] + 0.5   # one descent in the wavenumbers
    cases.append((U, b"sorted"))
    N = {k: v.copy() for k, v in S.items()}
    N["A"][777] = -1.0
    cases.append((N, b"invalid"))
    for lines, msg in cases:
        dl = {k: torch.from_numpy(v).cuda() for k, v in lines.items()}
        out = torch.full((len(conds), grid.n), 7.0, dtype=torch.float64, device="cuda:0")
        rc = _static_call(xc, dl, len(lines["nu"]), dE, dg, conds, grid, opts, out)
        assert rc == 1, rc
        assert msg in xc.lib().xc_last_error(), xc.lib().xc_last_error()
        assert bool(torch.all(out == 7.0))


def test_static_entry_rejects_sizes_beyond_its_limits(xc):
    dl = {k: torch.zeros(4, dtype=t, device="cuda:0") for k, t in
          (("nu", torch.float64), ("elower", torch.float32), ("A", torch.float32), ("gamma_ref", torch.float32),
           ("n_T", torch.float32), ("g_up", torch.int16), ("j_lo", torch.int16))}
    dE = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    dg = torch.ones(1, dtype=torch.int32, device="cuda:0")
    out = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    opts = xc.make_opts("voigt_w4", "fp32", 25.0)
    cond = [xc.make_condition(1000.0, 1.0)]
    rc = _static_call(xc, dl, (1 << 20) + 1, dE, dg, cond, xc.make_grid(0.0, 0.01, 4), opts, out)
    assert rc == 1 and b"limit" in xc.lib().xc_last_error()
    rc = _static_call(xc, dl, 4, dE, dg, cond, xc.make_grid(0.0, 0.01, (1 << 22) + 1), opts, out)
    assert rc == 1 and b"limit" in xc.lib().xc_last_error()
    rc = _static_call(xc, dl, 4, dE, dg, cond * 65, xc.make_grid(0.0, 0.01, 4), opts, out)
    assert rc == 1 and b"limit" in xc.lib().xc_last_error()
