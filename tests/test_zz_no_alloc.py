"""sgm_helmholtz_solve_noalloc against sgm_helmholtz_solve (GPU).

The allocation-free entry point serves callers that must not allocate device memory (a
program whose device memory belongs to one memory manager, or a latency-critical loop);
its elimination scratch is a fixed static device array shared by all calls.  This test
calls it twice in a row through the C ABI, with different right-hand sides, and checks
each result against the space-based solve within the parity tolerances of the other
solve tests (f64 1e-12, f32 2e-6 relative).  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

KIND = {"dirichlet": 1, "c2c": 3, "r2c": 4}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build, sgm
    build.build()
    return sgm


def _noalloc(sgm, kinds, sizes, prec, a, b, f, out):
    nd = len(kinds)
    k = (ctypes.c_int * nd)(*[KIND[x] for x in kinds])
    n = (ctypes.c_int64 * nd)(*sizes)
    st = sgm.lib().sgm_helmholtz_solve_noalloc(nd, k, n, None, sgm.PRECISION[prec], a, b,
                                               ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    sgm.check(st)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("kinds,sizes", [(["dirichlet", "c2c", "r2c"], [24, 40, 64]),
                                          (["dirichlet", "r2c"], [32, 33]),
                                          (["dirichlet", "c2c", "r2c"], [256, 64, 64])])
def test_noalloc_matches_space_solve(lib, kinds, sizes, prec, tol):
    sp = lib.Space(kinds, sizes, precision=prec)
    g = np.random.default_rng(5)
    for call, (a, b) in enumerate([(-1.0, 0.0), (1.0, -300.0)]):
        f = g.standard_normal(sp.spectral_shape) + 1j * g.standard_normal(sp.spectral_shape)
        f[sizes[0] - 2:] = 0
        fd = torch.from_numpy(f).to(sp.spectral_dtype).cuda()
        ref = sp.helmholtz_solve(a, b, fd)
        got = torch.full_like(fd, float("nan"))
        _noalloc(lib, kinds, sizes, prec, a, b, fd, got)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm((got - ref).to(torch.complex128)) /
               torch.linalg.vector_norm(ref.to(torch.complex128))).item()
        assert err < tol, (call, err)


def test_noalloc_rejects_sizes_past_the_limit(lib):
    f = torch.zeros(4100, 3, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.SgmError) as e:
        _noalloc(lib, ["dirichlet", "c2c"], [4100, 3], "f32", -1.0, 0.0, f, f)
    assert e.value.status == -2
