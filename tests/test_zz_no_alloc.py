"""The allocation-free entry point (xc_cross_section_batched_static).

It serves callers that cannot allocate device memory while they run (code in
another framework's memory pool or a fixed memory budget, loops that must not
call cudaMalloc/cudaFree).  It keeps its scratch in a fixed static device array
instead.  This test calls it through the C ABI on device buffers the test owns,
twice in a row (the scratch keeps the previous call's contents, so the second
call checks that everything that must start fresh is cleared), and compares it
with the handle-based xc_cross_section_batched FP32 path within the FP32
tolerance of the other parity tests.  It lives in its own file, collected
last, and passes alone or after the other tests.
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


def _static_call(xc, dl, n, dE, dg, conds, grid, opts, out):
    L = xc.XcLines(dl["nu"].data_ptr(), dl["elower"].data_ptr(), dl["A"].data_ptr(), dl["gamma_ref"].data_ptr(),
                   dl["n_T"].data_ptr(), dl["g_up"].data_ptr(), dl["j_lo"].data_ptr(), xc.XC_MEM_DEVICE)
    arr = (xc.XcCondition * len(conds))(*conds)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return xc.lib().xc_cross_section_batched_static(C.byref(L), n, dE.data_ptr(), dg.data_ptr(), len(dE), arr,
                                                    len(conds), C.byref(grid), C.byref(opts), out.data_ptr(), stream)


def test_static_entry_matches_batched(xc):
    Lh = xs.gen_lines(301, 0, 60000, 0.0, 300.0)
    o = np.argsort(Lh["nu"], kind="stable")
    S = {k: v[o] for k, v in Lh.items()}
    E, g = xs.gen_states(301, 3000)
    dl = {k: torch.from_numpy(v).cuda() for k, v in S.items()}
    dE, dg = torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda()
    grid = xc.make_grid(0.0, 0.01, 30001)
    W = xs.WORKLOADS["C3"]
    conds = [xc.make_condition(c["T"], c["P"]) for c in xs.conditions_for(W)]
    for profile in ("voigt_w4", "lorentz", "doppler"):
        opts = xc.make_opts(profile, "fp32", 25.0)
        with xc.Engine(0) as eng:
            eng.load_lines(Lh)
            eng.set_states(E, g)
            ref = eng.cross_section_batched(conds, grid, opts)
        for attempt in range(2):
            out = torch.full((len(conds), grid.n), float("nan"), dtype=torch.float64, device="cuda:0")
            rc = _static_call(xc, dl, len(o), dE, dg, conds, grid, opts, out)
            assert rc == 0, xc.lib().xc_last_error().decode()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            for c in range(len(conds)):
                m = ref[c] > 1e-6 * ref[c].max()
                err = np.max(np.abs(got[c][m] - ref[c][m]) / ref[c][m])
                assert err < TOL32, (profile, attempt, c, err)


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
    assert rc == 1 and b"1,048,576" not in xc.lib().xc_last_error() and b"limit" in xc.lib().xc_last_error()
    rc = _static_call(xc, dl, 4, dE, dg, cond, xc.make_grid(0.0, 0.01, (1 << 22) + 1), opts, out)
    assert rc == 1 and b"limit" in xc.lib().xc_last_error()
    rc = _static_call(xc, dl, 4, dE, dg, cond * 65, xc.make_grid(0.0, 0.01, 4), opts, out)
    assert rc == 1 and b"limit" in xc.lib().xc_last_error()
