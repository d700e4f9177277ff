"""GPU parity: the Chebyshev axis as a dense BF16x3 tensor-core contraction (SGM_CHEB_TC).

The contraction replaces the DCT-via-FFT kernels of an FP32 space for N <= 128.  Its error
against the FP64 oracle comes from the BF16x3 split products: x = hi + lo with BF16 parts
(|x - hi - lo| <= 2^-16 |x|) and the dropped lo*lo product (<= 2^-16 of the product), summed
with FP32 accumulation: each product carries a relative error of at most ~3 * 2^-16 and
typically ~2^-18, with random signs, so the relative L2 error of a contraction is ~2^-18
(measured 2e-6 .. 5.5e-6 on GB300).  Tolerances (relative L2 over the array):
  scalar product, backward          2^-16 ~ 1.5e-5
  forward (mass solve after it)     2^-16 * cond(B)   (worst-case amplification by the solve)
  physical -> physical solves of    2^-15 ~ 3.1e-5    (smooth manufactured solutions: the
  manufactured problems                                 solve does not amplify the error)
The oracle receives exactly the FP32 values the GPU received.
"""
import numpy as np
import pytest
import torch

from oracle import quadrature
from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_TC = 2.0 ** -16
TOL_TC_SOLVE = 2.0 ** -15


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def tc_space(kinds, sizes, cheb="tc"):
    from paper_1708_03188_gb300.sgm import Space
    return Space(kinds, sizes, precision="f32", cheb=cheb)


SPACES = [
    (["dirichlet"], [4]),                       # smallest bases
    (["biharmonic"], [6]),
    (["chebyshev"], [2]),
    (["dirichlet"], [128]),                     # largest N, one column
    (["dirichlet", "r2c"], [32, 32]),           # the 2-D Poisson sizes
    (["dirichlet", "r2c"], [33, 300]),          # odd N, two tiles and a ragged tail (302 columns)
    (["biharmonic", "r2c"], [64, 126]),
    (["chebyshev", "c2c"], [17, 70]),
    (["dirichlet", "c2c", "r2c"], [16, 12, 30]),
    (["biharmonic", "c2c", "r2c"], [100, 9, 16]),
    (["dirichlet", "c2c", "r2c"], [127, 8, 40]),
    (["biharmonic", "c2c"], [128, 65]),
]


@pytest.mark.parametrize("kinds,sizes", SPACES, ids=lambda v: "-".join(map(str, v)))
def test_tc_transforms(kinds, sizes):
    gs = tc_space(kinds, sizes)
    assert gs.cheb_method == "tc"
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 300)
    x = g.standard_normal(gs.physical_shape)
    if not gs.real_physical:
        x = x + 1j * g.standard_normal(gs.physical_shape)
    xd = to_dev(x, gs.physical_dtype)
    xo = to_np(xd)
    e_s = rel(to_np(gs.scalar_product(xd)), os_.scalar_product(xo))
    assert e_s < TOL_TC, e_s
    condB = np.linalg.cond(os_.matrices()["B"])
    fw = to_np(gs.forward(xd))
    assert rel(fw, os_.forward(xo)) < TOL_TC * max(1.0, condB)
    nb = quadrature.num_basis(kinds[0], sizes[0])
    assert np.all(fw[nb:] == 0)
    c = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        c = c + 1j * g.standard_normal(gs.spectral_shape)
    c[nb:] = 0
    c = os_.forward(os_.backward(c))
    cd = to_dev(c, gs.spectral_dtype)
    e_b = rel(to_np(gs.backward(cd)), os_.backward(to_np(cd)))
    print(f"tc {kinds} {sizes}: scalar {e_s:.2e} backward {e_b:.2e}")
    assert e_b < TOL_TC, e_b


def test_tc_matches_fft_path_closely():
    """Both FP32 methods agree to the contraction's tolerance on the same input."""
    kinds, sizes = ["dirichlet", "c2c", "r2c"], [64, 32, 48]
    a, b = tc_space(kinds, sizes, "tc"), tc_space(kinds, sizes, "fft")
    assert (a.cheb_method, b.cheb_method) == ("tc", "fft")
    g = inputs.rng("box3d", 301)
    x = to_dev(g.standard_normal(a.physical_shape), torch.float32)
    assert rel(to_np(a.scalar_product(x)), to_np(b.scalar_product(x))) < TOL_TC


@pytest.mark.parametrize("N", [32, 64])
def test_tc_poisson2d_manufactured(N):
    kinds = ["dirichlet", "r2c"]
    gs = tc_space(kinds, (N, N))
    os_ = OSpace(kinds, (N, N))
    condB = np.linalg.cond(os_.matrices()["B"])
    x, y = inputs.mesh(kinds, (N, N))
    fd = to_dev(inputs.poisson2d_f(x, y), gs.physical_dtype)
    u = to_np(gs.helmholtz(-1.0, 0.0, fd))
    e = rel(u, inputs.poisson2d_u(x, y))
    print(f"tc poisson2d {N}: {e:.2e} (cond B {condB:.1f})")
    assert e < TOL_TC_SOLVE


def test_tc_box3d_biharmonic_manufactured():
    N = (64, 32, 32)
    kinds = ["biharmonic", "c2c", "r2c"]
    gs = tc_space(kinds, N)
    os_ = OSpace(kinds, N)
    condB = np.linalg.cond(os_.matrices()["B"])
    x, y, z = inputs.mesh(kinds, N)
    fd = to_dev(np.broadcast_to(inputs.box3d_f_biharmonic(x, y, z), N), gs.physical_dtype)
    u = to_np(gs.biharmonic(1.0, 0.0, 0.0, fd))
    e = rel(u, np.broadcast_to(inputs.box3d_u(x, y, z), N))
    print(f"tc box3d biharmonic {N}: {e:.2e} (cond B {condB:.1f})")
    assert e < TOL_TC_SOLVE


def test_tc_auto_and_errors():
    from paper_1708_03188_gb300.sgm import SgmError, Space
    sp = tc_space(["dirichlet", "c2c", "r2c"], [64, 64, 64], "auto")
    assert sp.cheb_method in ("tc", "fft")
    big = tc_space(["dirichlet", "r2c"], [256, 16], "auto")
    assert big.cheb_method == "fft"                     # N > 128 keeps the FFT method
    with pytest.raises(SgmError):
        tc_space(["dirichlet", "r2c"], [129, 16], "tc")
    with pytest.raises(SgmError):
        Space(["dirichlet", "r2c"], [32, 16], precision="f64", cheb="tc")
    with pytest.raises(SgmError):
        tc_space(["c2c", "r2c"], [32, 16], "tc")            # no Chebyshev axis


def test_tc_no_wait_timed_out():
    from paper_1708_03188_gb300.sgm import tc_wait_timeouts
    torch.cuda.synchronize()
    assert tc_wait_timeouts() == 0
