"""The allocation-free small adjoint (ftcg_adjoint_small_noalloc) against the plan-based
ftcg_adjoint, through the C ABI.

This entry point is for callers that cannot allocate device memory (code running under stream
capture, fixed-footprint real-time loops, frameworks that own the memory pool). Its scratch is a
set of fixed device arrays shared by every call, so the test makes two calls in a row with
different inputs and checks each against the plan-based result, which also shows that the first
call's contents do not leak into the second. The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import sasgen

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as pkg
    return pkg


def _noalloc(F, lam, v, alpha, N, sigma, w, out):
    import torch
    L = F.lib()
    st = L.ftcg_adjoint_small_noalloc(
        ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(v.data_ptr()),
        ctypes.c_void_p(alpha.data_ptr()) if alpha is not None else None,
        int(lam.shape[0]), N, sigma, w, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_plan_adjoint_twice(F):
    import torch
    p = sasgen.tiny()
    lam = torch.from_numpy(p.lam).cuda()
    v1 = torch.from_numpy(sasgen.values_for(p).astype(np.complex64)).cuda()
    rng = np.random.default_rng(3)
    v2 = torch.from_numpy((rng.standard_normal(p.M) + 1j * rng.standard_normal(p.M))
                          .astype(np.complex64)).cuda()
    alpha = torch.from_numpy(rng.uniform(0.3, 1.7, p.M)).cuda()
    with F.Plan(lam, p.N, p.sigma, p.w) as plan:
        plan.set_weights(alpha)
        ref1 = plan.adjoint(v1).cpu().numpy()
        plan.set_weights(None)
        ref2 = plan.adjoint(v2).cpu().numpy()
    out1 = torch.empty((p.N, p.N), dtype=torch.complex64, device="cuda")
    out2 = torch.empty((p.N, p.N), dtype=torch.complex64, device="cuda")
    assert _noalloc(F, lam, v1, alpha, p.N, p.sigma, p.w, out1) == 0
    assert _noalloc(F, lam, v2, None, p.N, p.sigma, p.w, out2) == 0
    torch.cuda.synchronize()
    assert rel_l2(out1.cpu().numpy(), ref1) < TOL
    assert rel_l2(out2.cpu().numpy(), ref2) < TOL


def test_noalloc_rejects_large_grid(F):
    import torch
    lam = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    v = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.empty((512, 512), dtype=torch.complex64, device="cuda")
    assert _noalloc(F, lam, v, None, 512, 2.0, 8, out) == 4      # G = 1024 > 512
    assert b"exceeds" in F.lib().ftcg_last_error()


def test_noalloc_at_the_size_limit(F):
    """G = sigma N = 512, the largest grid the fixed scratch holds (N = 256, sigma = 2)."""
    import torch
    lam_np, v_np = sasgen.random_case(61, 20000, 256, 2.0, 8, 256)
    lam = torch.from_numpy(lam_np).cuda()
    v = torch.from_numpy(v_np.astype(np.complex64)).cuda()
    with F.Plan(lam, 256, 2.0, 8) as plan:
        ref = plan.adjoint(v).cpu().numpy()
    out = torch.empty((256, 256), dtype=torch.complex64, device="cuda")
    assert _noalloc(F, lam, v, None, 256, 2.0, 8, out) == 0
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref) < TOL



def test_noalloc_captured_in_cuda_graph(F):
    """The entry point's main use: a call captured in a CUDA graph (after one warm call) and
    replayed with new contents of the same value buffer; each replay against the plan-based
    adjoint of those values."""
    import torch
    p = sasgen.tiny()
    lam = torch.from_numpy(p.lam).cuda()
    rng = np.random.default_rng(11)
    alpha = torch.from_numpy(rng.uniform(0.3, 1.7, p.M)).cuda()
    v = torch.zeros(p.M, dtype=torch.complex64, device="cuda")
    out = torch.empty((p.N, p.N), dtype=torch.complex64, device="cuda")
    assert _noalloc(F, lam, v, alpha, p.N, p.sigma, p.w, out) == 0        # warm call
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = _noalloc(F, lam, v, alpha, p.N, p.sigma, p.w, out)
    assert st == 0
    with F.Plan(lam, p.N, p.sigma, p.w) as plan:
        plan.set_weights(alpha)
        for seed in (1, 2):
            r = np.random.default_rng(seed)
            x = (r.standard_normal(p.M) + 1j * r.standard_normal(p.M)).astype(np.complex64)
            v.copy_(torch.from_numpy(x))
            g.replay()
            torch.cuda.synchronize()
            ref = plan.adjoint(torch.from_numpy(x).cuda()).cpu().numpy()
            assert rel_l2(out.cpu().numpy(), ref) < TOL
