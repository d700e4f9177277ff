"""sgm_helmholtz_solve_noalloc (GPU): the Shen-Dirichlet Helmholtz solve that allocates nothing.

Who calls it: code that must not allocate device memory itself, such as a program whose device
memory belongs to one memory manager (a framework's caching allocator, or a budget claimed up
front) or a latency-critical loop that cannot afford the time or the failure of a cudaMalloc.
Its elimination scratch is a fixed static device array shared by all calls.

Checks, each through the C ABI on two calls in a row with different right-hand sides (the
second call reuses the array the first one left behind):
  - against sgm_helmholtz_solve on a space built from the same arguments, within the parity
    tolerances of the other solve tests (FP64 1e-12, FP32 2e-6 relative);
  - against the FP64 oracle's dense LU of each column's Galerkin system (small sizes);
  - the 1-D case (real spectral data), the largest N (2048) and argument rejections.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle.space import Space as OracleSpace

pytestmark = pytest.mark.gpu

KIND = {"dirichlet": 1, "c2c": 3, "r2c": 4}
CASES = [(["dirichlet", "c2c", "r2c"], [24, 40, 64]),
         (["dirichlet", "r2c"], [32, 33]),
         (["dirichlet"], [64]),
         (["dirichlet", "c2c", "r2c"], [256, 64, 64]),
         (["dirichlet", "c2c"], [2048, 8])]
COEFFS = [(-1.0, 0.0), (1.0, -300.0)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build, sgm
    build.build()
    return sgm


def _noalloc(sgm, kinds, sizes, prec, a, b, f, out, domain=None):
    nd = len(kinds)
    k = (ctypes.c_int * nd)(*[KIND[x] for x in kinds])
    n = (ctypes.c_int64 * nd)(*sizes)
    dom = None if domain is None else (ctypes.c_double * (2 * nd))(*[v for pair in domain for v in pair])
    st = sgm.lib().sgm_helmholtz_solve_noalloc(nd, k, n, dom, sgm.PRECISION[prec], a, b,
                                               ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    sgm.check(st)


def _rhs(g, shape, N, real):
    f = g.standard_normal(shape) if real else g.standard_normal(shape) + 1j * g.standard_normal(shape)
    f[N - 2:] = 0
    return f


def _rel(x, y):
    return float(np.linalg.norm((x - y).ravel()) / np.linalg.norm(y.ravel()))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("kinds,sizes", CASES)
def test_noalloc_matches_space_solve_and_oracle(lib, kinds, sizes, prec, tol):
    sp = lib.Space(kinds, sizes, precision=prec)
    g = np.random.default_rng(5)
    real = len(kinds) == 1
    oracle = OracleSpace(kinds, sizes) if sizes[0] <= 256 and np.prod(sp.spectral_shape) <= 256 * 64 * 33 else None
    for call, (a, b) in enumerate(COEFFS):
        f = _rhs(g, sp.spectral_shape, sizes[0], real)
        fd = torch.from_numpy(f).to(sp.spectral_dtype).cuda()
        ref = sp.helmholtz_solve(a, b, fd)
        got = torch.full_like(fd, float("nan"))
        _noalloc(lib, kinds, sizes, prec, a, b, fd, got)
        torch.cuda.synchronize()
        got_h = got.cpu().numpy().astype(np.complex128)
        err = _rel(got_h, ref.cpu().numpy().astype(np.complex128))
        assert err < tol, ("against sgm_helmholtz_solve", call, err)
        if oracle is not None:
            uo = oracle.helmholtz(a, b, fd.cpu().numpy().astype(np.complex128))
            e_o = _rel(got_h, uo)
            assert e_o < tol, ("against the oracle", call, e_o)
        assert np.all(got_h[sizes[0] - 2:] == 0)
    sp.close()


def test_noalloc_rejects_sizes_past_the_limit(lib):
    f = torch.zeros(2049, 3, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.SgmError) as e:
        _noalloc(lib, ["dirichlet", "c2c"], [2049, 3], "f32", -1.0, 0.0, f, f)
    assert e.value.status == -2


def test_noalloc_rejects_arguments_the_space_rejects(lib):
    f = torch.zeros(16, 9, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.SgmError) as e:   # the Chebyshev axis lives on [-1, 1] only
        _noalloc(lib, ["dirichlet", "r2c"], [16, 16], "f32", -1.0, 0.0, f, f, domain=[(0.0, 2.0), (0.0, 6.0)])
    assert e.value.status == -3
    g = torch.zeros(16, 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.SgmError) as e:   # an R2C axis needs M >= 2
        _noalloc(lib, ["dirichlet", "r2c"], [16, 1], "f32", -1.0, 0.0, g, g)
    assert e.value.status == -2
