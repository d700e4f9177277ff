"""GPU parity: Legendre bases on axis 0 (dense transforms, banded FP64 solves) against the oracle.

Tolerances (relative L2 over the array):
  f64 transforms            1e-12   dense FP64 sums of at most 1024 terms
  f32 transforms            4e-6    dense FP32 sums: ~sqrt(N) 2^-24 per output, N <= 100 here
  forward (mass solve)      the transform tolerance times cond(B), as for the Chebyshev bases
  f64 solves                1e-12   (well-conditioned systems; FP64 elimination)
  f32 solves                2e-6    FP64 elimination on FP32 data, rounded once
The oracle receives exactly the values the GPU received.
"""
import numpy as np
import pytest
import torch

from oracle import quadrature
from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 4e-6}
TOL_SOLVE = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def gspace(kinds, sizes, prec):
    from paper_1708_03188_gb300.sgm import Space
    return Space(kinds, sizes, precision=prec)


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


SPACES = [
    (["legendre"], [2]),                                   # smallest bases
    (["legendre_dirichlet"], [4]),
    (["legendre_biharmonic"], [6]),
    (["legendre_dirichlet"], [97]),                        # two row tiles, the second ragged
    (["legendre_biharmonic", "r2c"], [40, 30]),
    (["legendre", "c2c"], [17, 9]),
    (["legendre_dirichlet", "c2c", "r2c"], [24, 10, 18]),
    (["legendre_biharmonic", "c2c", "r2c"], [70, 6, 301]),  # 1812 real columns: 29 column tiles
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", SPACES, ids=lambda v: "-".join(map(str, v)))
def test_legendre_transforms(kinds, sizes, prec):
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 800 + sizes[0])
    x = g.standard_normal(gs.physical_shape)
    if not gs.real_physical:
        x = x + 1j * g.standard_normal(gs.physical_shape)
    xd = to_dev(x, gs.physical_dtype)
    xo = to_np(xd)
    assert rel(to_np(gs.scalar_product(xd)), os_.scalar_product(xo)) < TOL[prec]
    cond = 1.0 if kinds[0] == "legendre" else np.linalg.cond(os_.matrices()["B"])
    fw = to_np(gs.forward(xd))
    assert rel(fw, os_.forward(xo)) < TOL[prec] * max(1.0, cond)
    nb = quadrature.num_basis(kinds[0], sizes[0])
    assert np.all(fw[nb:] == 0)
    c = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        c = c + 1j * g.standard_normal(gs.spectral_shape)
    c[nb:] = 0
    c = os_.forward(os_.backward(c))                      # consistent Hermitian planes
    cd = to_dev(c, gs.spectral_dtype)
    assert rel(to_np(gs.backward(cd)), os_.backward(to_np(cd))) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", [(["legendre_dirichlet"], [40]), (["legendre_dirichlet", "r2c"], [32, 33]),
                                         (["legendre_dirichlet", "c2c", "r2c"], [20, 12, 16])],
                         ids=lambda v: "-".join(map(str, v)))
@pytest.mark.parametrize("a,b", [(-1.0, 0.0), (1.0, -300.0), (0.0, 1.0)])
def test_legendre_helmholtz_solve(kinds, sizes, prec, a, b):
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 850)
    f = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        f = f + 1j * g.standard_normal(gs.spectral_shape)
    fd = to_dev(f, gs.spectral_dtype)
    assert rel(to_np(gs.helmholtz_solve(a, b, fd)), os_.helmholtz(a, b, to_np(fd))) < TOL_SOLVE[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", [(["legendre_biharmonic"], [40]), (["legendre_biharmonic", "r2c"], [34, 18]),
                                         (["legendre_biharmonic", "c2c", "r2c"], [24, 8, 12])],
                         ids=lambda v: "-".join(map(str, v)))
@pytest.mark.parametrize("a,b,c", [(1.0, 0.0, 0.0), (1.3, -0.4, 2.0), (0.0, 0.0, 1.0)])
def test_legendre_biharmonic_solve(kinds, sizes, prec, a, b, c):
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 860)
    f = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        f = f + 1j * g.standard_normal(gs.spectral_shape)
    fd = to_dev(f, gs.spectral_dtype)
    got = to_np(gs.biharmonic_solve(a, b, c, fd))
    assert rel(got, os_.biharmonic(a, b, c, to_np(fd))) < TOL_SOLVE[prec]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("kind", ["legendre_dirichlet", "legendre_biharmonic"])
def test_legendre_box3d_manufactured(prec, tol, kind):
    N = (24, 16, 16)
    kinds = [kind, "c2c", "r2c"]
    gs = gspace(kinds, N, prec)
    x, y, z = inputs.mesh(kinds, N)
    if kind == "legendre_dirichlet":
        f = to_dev(np.broadcast_to(inputs.box3d_f_poisson(x, y, z), N), gs.physical_dtype)
        u = to_np(gs.helmholtz(-1.0, 0.0, f))
    else:
        f = to_dev(np.broadcast_to(inputs.box3d_f_biharmonic(x, y, z), N), gs.physical_dtype)
        u = to_np(gs.biharmonic(1.0, 0.0, 0.0, f))
    assert rel(u, np.broadcast_to(inputs.box3d_u(x, y, z), N)) < tol


def test_legendre_errors():
    from paper_1708_03188_gb300.sgm import SgmError, Space
    with pytest.raises(SgmError):
        Space(["legendre_dirichlet", "r2c"], [1025, 8], precision="f64")
    with pytest.raises(SgmError):
        Space(["legendre_dirichlet", "r2c"], [129, 8], precision="f32", cheb="tc")   # N <= 128 on the tensor cores
    with pytest.raises(SgmError):
        Space(["legendre_dirichlet", "r2c"], [32, 8], precision="f64", cheb="tc")
    with pytest.raises(SgmError):   # at most one polynomial axis
        Space(["legendre", "legendre_dirichlet"], [8, 8], precision="f64")
    # a Legendre axis after a Fourier axis is the axes option of Sec. 4: a permuted view
    ps = Space(["c2c", "legendre"], [8, 6], precision="f64")
    assert ps.spectral_shape == (8, 6)
    ps.close()
    gs = gspace(["legendre_biharmonic", "c2c"], [16, 8], "f64")
    x = torch.zeros(gs.spectral_shape, dtype=gs.spectral_dtype, device="cuda")
    with pytest.raises(SgmError):
        gs.helmholtz_solve(-1.0, 0.0, x)
    assert gs.chebyshev_space().kinds == ("legendre", "c2c")


TOL_TC = 2.0 ** -16      # BF16x3 split products, FP32 accumulation (as for the Chebyshev contraction)


@pytest.mark.parametrize("kinds,sizes", [(["legendre"], [2]), (["legendre_dirichlet"], [128]),
                                         (["legendre_biharmonic", "r2c"], [64, 126]),
                                         (["legendre_dirichlet", "c2c", "r2c"], [33, 12, 30])],
                         ids=lambda v: "-".join(map(str, v)))
def test_legendre_tensor_core_transforms(kinds, sizes):
    from paper_1708_03188_gb300.sgm import Space
    gs = Space(kinds, sizes, precision="f32", cheb="tc")
    assert gs.cheb_method == "tc"
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 870 + sizes[0])
    x = g.standard_normal(gs.physical_shape)
    if not gs.real_physical:
        x = x + 1j * g.standard_normal(gs.physical_shape)
    xd = to_dev(x, gs.physical_dtype)
    xo = to_np(xd)
    assert rel(to_np(gs.scalar_product(xd)), os_.scalar_product(xo)) < TOL_TC
    cond = 1.0 if kinds[0] == "legendre" else np.linalg.cond(os_.matrices()["B"])
    assert rel(to_np(gs.forward(xd)), os_.forward(xo)) < TOL_TC * max(1.0, cond)
    nb = quadrature.num_basis(kinds[0], sizes[0])
    c = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        c = c + 1j * g.standard_normal(gs.spectral_shape)
    c[nb:] = 0
    c = os_.forward(os_.backward(c))
    cd = to_dev(c, gs.spectral_dtype)
    assert rel(to_np(gs.backward(cd)), os_.backward(to_np(cd))) < TOL_TC
    auto = Space(kinds, sizes, precision="f32", cheb="auto")
    assert auto.cheb_method in ("tc", "dense")
