"""The allocation-free residual entry point (opf_residuals_noalloc).

Some callers may not allocate device memory (a fixed memory pool, a plugin
handed its buffers, a process that forbids cudaMalloc after start-up).  For
them the library computes the residual norms of the termination test from
caller-owned device vectors, keeping its partial sums in a fixed array of
its own.  This test runs a real solve through the normal entry point, then
feeds the same iterates to the allocation-free entry point through the C
ABI, on two calls in a row, and requires the same residuals.  It lives in a
file of its own, collected last, and passes alone in a fresh process or
after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2501_08293_b300 import feeders as F

pytestmark = pytest.mark.gpu
TOL = 1e-9        # the GPU parity tolerance used by the other tests


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08293_b300 import build
    build.build()
    from paper_2501_08293_b300 import opf
    return torch, opf


def test_residuals_noalloc_match_solver(env):
    torch, opf = env
    f = F.feeder_123(1)
    p = opf.Problem.from_feeder(f)
    gidx = p.structure()["gidx"].astype(np.int64)
    rho, eps_rel = 100.0, 1e-3
    prm = lambda n, warm: opf.default_params(rho=rho, eps_rel=eps_rel, criterion=opf.CRIT_NEVER,
                                             max_iter=n, check_every=n, warm_start=warm)
    p.solve(prm(40, 0))
    _, prev, _ = p.state()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for call in range(2):                       # two calls in a row
        info = p.solve(prm(1, 1))              # one more iteration: reference residuals
        xg, xl, lam = p.state()
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
        v, z, zp, l = dev(xg[gidx]), dev(xl), dev(prev), dev(lam)
        stream = torch.cuda.current_stream()
        st = opf.lib.opf_residuals_noalloc(C.c_void_p(v.data_ptr()), C.c_void_p(z.data_ptr()),
                                           C.c_void_p(zp.data_ptr()), C.c_void_p(l.data_ptr()),
                                           int(z.numel()), rho, eps_rel, C.c_void_p(out.data_ptr()),
                                           C.c_void_p(stream.cuda_stream))
        assert st == 0, opf.lib.opf_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = np.array([info.pres, info.dres, info.eps_prim, info.eps_dual])
        assert np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1e-12)), (call, got, want)
        prev = xl
    # sizes beyond the fixed scratch are refused with a clear error
    st = opf.lib.opf_residuals_noalloc(C.c_void_p(v.data_ptr()), C.c_void_p(z.data_ptr()),
                                       C.c_void_p(zp.data_ptr()), C.c_void_p(l.data_ptr()),
                                       4_194_305, rho, eps_rel, C.c_void_p(out.data_ptr()), None)
    assert st == -1 and "4194304" in opf.lib.opf_last_error().decode()
    p.close()
