"""The allocation-free dense apply, for callers that must not call cudaMalloc
(real-time loops and plugin hosts that reserve device memory up front).

It is checked through the C ABI on two calls in a row against the scene-based
global solve (flash_global_apply, FP32 path) and against a float64 product
on the host, also with a non-symmetric matrix (the call must return
Ainv * rhs, not its transpose applied).  The second call is smaller than the
first, so stale scratch contents from the first call would show up in its
padding.  Collected last on purpose: it holds a fixed
__device__ scratch array and should run after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu

REL_TOL = 2e-5   # the FP32 global-apply tolerance of the other GPU tests


def _noalloc(lib, Ainv, n, m, rhs, out, stream):
    f = lib.flash_dense_apply_noalloc
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int32
    return f(C.c_void_p(Ainv.data_ptr()), n, m, C.c_void_p(rhs.data_ptr()), C.c_void_p(out.data_ptr()), stream)


def test_noalloc_apply_matches_global_apply(cuda):
    import torch
    from paper_2604_17513_gb300 import flash
    lib = flash.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(11)
    for m in (6, 2):   # two calls in a row, the second smaller
        sc = scenes.cloth_drop(n_envs=m)
        n = sc.n_verts
        sim = flash.Sim(sc, solve=flash.SOLVE_F32)
        rhs = torch.from_numpy((rng.normal(size=(m * n, 3)) * 1e-3).astype(np.float32)).to(cuda)
        ref = sim.global_apply(0, m, rhs)
        # the caller's own A^-1 (here from the oracle's system matrix)
        A = oracle.Mesh.from_scene(sc).matrix()
        Ainv = torch.from_numpy(np.linalg.inv(A).astype(np.float32)).to(cuda)
        out = torch.full((m * n, 3), float("nan"), dtype=torch.float32, device=cuda)
        assert _noalloc(lib, Ainv, n, m, rhs, out, stream) == flash.OK
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err < REL_TOL, (m, err)
        host = np.einsum("ij,ejc->eic", Ainv.cpu().numpy().astype(np.float64),
                         rhs.cpu().numpy().astype(np.float64).reshape(m, n, 3))
        err64 = np.abs(out.cpu().numpy().reshape(m, n, 3) - host).max() / np.abs(host).max()
        assert err64 < REL_TOL, (m, err64)


def test_noalloc_apply_non_symmetric_matches_float64(cuda):
    """out = Ainv * rhs for a random non-symmetric [n][n] matrix, against the
    float64 host product, on two calls in a row (the second smaller)."""
    import torch
    from paper_2604_17513_gb300 import flash
    lib = flash.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(12)
    for n, m in ((300, 40), (130, 3)):
        M = rng.normal(size=(n, n)) + 4.0 * np.eye(n) + 2.0 * np.triu(rng.normal(size=(n, n)), 1)
        assert np.abs(M - M.T).max() > 1.0
        Mf = M.astype(np.float32)
        rhs = rng.normal(size=(m, n, 3)).astype(np.float32)
        ref = np.einsum("ij,ejc->eic", Mf.astype(np.float64), rhs.astype(np.float64))
        out = torch.full((m * n, 3), float("nan"), dtype=torch.float32, device=cuda)
        code = _noalloc(lib, torch.from_numpy(Mf).to(cuda), n, m, torch.from_numpy(rhs.reshape(-1, 3)).to(cuda),
                        out, stream)
        assert code == flash.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(m, n, 3).astype(np.float64)
        # FP32 products over n terms: |err| <= n u sum_j |M_ij| |rhs_j|
        bound = n * 2.0 ** -23 * np.einsum("ij,ejc->eic", np.abs(Mf), np.abs(rhs).astype(np.float64))
        assert np.all(np.abs(got - ref) <= bound), (n, m, np.abs(got - ref).max())
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < REL_TOL, (n, m, err)


def test_noalloc_rejects_sizes_beyond_scratch(cuda):
    import torch
    from paper_2604_17513_gb300 import flash
    lib = flash.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    small = torch.zeros((4, 3), dtype=torch.float32, device=cuda)
    code = _noalloc(lib, small, 600, 1, small, small, stream)          # n > 512
    assert code == flash.EINVAL and b"scratch" in lib.flash_last_error()
    code = _noalloc(lib, small, 128, 300, small, small, stream)        # m > 256
    assert code == flash.EINVAL
