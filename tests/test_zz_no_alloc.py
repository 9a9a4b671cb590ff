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


@pytest.mark.parametrize("n", [0, 1, 2048 * 8 * 3 + 777, 2048 * 8 * 256])
def test_residuals_noalloc_sizes(env, n):
    """Seeded random vectors at the edges of the fixed scratch: no locals,
    one, a partial last CTA, and the largest size it supports (every slot
    in use).  Two calls in a row on different data; each is compared with
    numpy FP64 norms at 1e-12 relative."""
    torch, opf = env
    rng = np.random.default_rng(1234 + n)
    rho, eps_rel = 37.5, 2e-3
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        a = [rng.standard_normal(n) * s for s in (1.0, 1.0, 0.5, 3.0)]
        v, z, zp, l = a[0], a[0] + 1e-3 * a[1], a[0] + 1e-3 * a[1] + 1e-4 * a[2], a[3]
        d = [torch.from_numpy(x).to("cuda") if n else torch.zeros(1, dtype=torch.float64, device="cuda")
             for x in (v, z, zp, l)]
        st = opf.lib.opf_residuals_noalloc(*[C.c_void_p(t.data_ptr()) for t in d], n, rho, eps_rel,
                                           C.c_void_p(out.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, opf.lib.opf_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        nrm = lambda x: float(np.sqrt(np.sum(x * x)))
        want = np.array([nrm(v - z), rho * nrm(z - zp), eps_rel * max(nrm(v), nrm(z)), eps_rel * nrm(l)])
        assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (n, call, got, want)
