"""The allocation-free dense apply, for callers that must not call cudaMalloc
(real-time loops and plugin hosts that reserve device memory up front).

It is checked through the C ABI against the scene-based global solve
(flash_global_apply, FP32 path) on two calls in a row; the second call is
smaller than the first, so stale scratch contents from the first call would
show up in its padding.  Collected last on purpose: it holds a fixed
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
