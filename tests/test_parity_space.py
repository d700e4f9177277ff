"""GPU parity: libsgm transforms and solves against the FP64 oracle.

Tolerances (relative L2 over the whole array unless stated):
  f64 transforms                  1e-12
  f32 transforms                  4e-6   (FP32 FFT/DCT: ~log2(N) * 2^-24 per pass, a few passes)
  f64 solves                      max(1e-12, 32 * 2^-53 * cond), cond = largest condition
                                  number of the column systems, plus a per-column normwise
                                  backward error <= 16 * 2^-53
  f32 solves (FP64 elimination)   2e-6   (inputs and outputs rounded to FP32 once)
The oracle receives exactly the values the GPU received (f32 inputs are widened).
"""
import numpy as np
import pytest
import torch

from oracle import galerkin, quadrature
from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def gspace(kinds, sizes, prec, domain=None):
    from paper_1708_03188_gb300.sgm import Space
    return Space(kinds, sizes, domain=domain, precision=prec)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def random_physical(sp, item):
    g = inputs.rng("box3d", 100 + item)
    x = g.standard_normal(sp.physical_shape)
    if not sp.real_physical:
        x = x + 1j * g.standard_normal(sp.physical_shape)
    return x


def random_spectral(osp, gsp, item):
    """Random coefficients on the valid index set, made consistent (Hermitian planes of an
    R2C axis) by one oracle backward + forward round trip."""
    g = inputs.rng("box3d", 200 + item)
    c = g.standard_normal(gsp.spectral_shape)
    if not gsp.real_spectral:
        c = c + 1j * g.standard_normal(gsp.spectral_shape)
    if osp.has_cheb:
        c[quadrature.num_basis(osp.kinds[0], osp.sizes[0]):] = 0
    return osp.forward(osp.backward(c))


SPACES = [
    (["dirichlet"], [32]),
    (["biharmonic"], [33]),
    (["chebyshev"], [17]),
    (["dirichlet", "r2c"], [32, 33]),          # Sec. 4, Fig. poisson2D sizes
    (["dirichlet", "r2c"], [20, 64]),
    (["biharmonic", "r2c"], [34, 18]),
    (["chebyshev", "c2c"], [9, 7]),
    (["dirichlet", "c2c"], [12, 10]),
    (["dirichlet", "c2c", "r2c"], [12, 10, 18]),
    (["biharmonic", "c2c", "r2c"], [32, 33, 34]),   # Sec. 4 biharmonic sizes
    (["dirichlet", "c2c", "r2c"], [24, 40, 64]),
    (["c2c"], [15]),
    (["r2c"], [16]),
    (["r2c"], [15]),
    (["c2c", "c2c"], [12, 10]),
    (["c2c", "r2c"], [9, 16]),
    (["c2c", "c2c", "c2c"], [6, 8, 5]),
    (["dirichlet", "r2c"], [4, 2]),            # smallest sizes
    (["biharmonic", "c2c"], [6, 1]),
    # lengths with compile-time FFT kernels (2^a and 3 * 2^a), several tiles plus ragged tails
    (["dirichlet", "c2c", "r2c"], [64, 256, 128]),
    (["biharmonic", "c2c", "r2c"], [128, 32, 64]),
    (["c2c", "c2c"], [768, 48]),
    (["c2c", "r2c"], [192, 1536]),
    (["chebyshev", "c2c"], [256, 19]),
    (["dirichlet", "c2c"], [512, 24]),
    (["biharmonic"], [384]),
    # equal Fourier lengths: the eliminations group the columns (+-a, b), (+-b, a)
    (["dirichlet", "c2c", "r2c"], [24, 16, 16]),
    (["biharmonic", "c2c", "r2c"], [20, 9, 9]),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", SPACES, ids=lambda v: "-".join(map(str, v)))
def test_transforms(kinds, sizes, prec):
    tol = 1e-12 if prec == "f64" else 4e-6
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    x = random_physical(gs, 0)
    xd = to_dev(x, gs.physical_dtype)
    xo = to_np(xd)                      # exactly the values the GPU sees
    assert rel(to_np(gs.scalar_product(xd)), os_.scalar_product(xo)) < tol
    # the forward transform ends with the mass-matrix solve: errors of the scalar product
    # are amplified by at most cond(B)
    condB = np.linalg.cond(os_.matrices()["B"]) if os_.has_cheb else 1.0
    assert rel(to_np(gs.forward(xd)), os_.forward(xo)) < tol * max(1.0, condB)
    c = random_spectral(os_, gs, 1)
    cd = to_dev(c, gs.spectral_dtype)
    co = to_np(cd)
    assert rel(to_np(gs.backward(cd)), os_.backward(co)) < tol
    # trailing Shen rows are written as zero
    if os_.has_cheb:
        nb = quadrature.num_basis(kinds[0], sizes[0])
        assert np.all(to_np(gs.forward(xd))[nb:] == 0)


def _column_systems(os_, build):
    k2 = np.atleast_1d(os_.kappa2()).ravel() if len(os_.sizes) > 1 else np.zeros(1)
    return [build(v) for v in k2]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", [(["dirichlet"], [40]), (["dirichlet", "r2c"], [32, 33]),
                                          (["dirichlet", "c2c", "r2c"], [24, 40, 64]),
                                          (["dirichlet", "c2c"], [65, 9]),
                                          (["dirichlet", "c2c", "r2c"], [24, 16, 16]),
                                          (["dirichlet", "c2c", "r2c"], [16, 9, 9])])
@pytest.mark.parametrize("a,b", [(-1.0, 0.0), (1.0, -300.0), (0.5, 2.0), (0.0, 1.0)])
def test_helmholtz_solve(kinds, sizes, prec, a, b):
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("poisson2d", 11)
    f = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        f = f + 1j * g.standard_normal(gs.spectral_shape)
    f[sizes[0] - 2:] = 0
    fd = to_dev(f, gs.spectral_dtype)
    fo = to_np(fd)
    got = to_np(gs.helmholtz_solve(a, b, fd))
    ref = os_.helmholtz(a, b, fo)
    mats = os_.matrices()
    systems = _column_systems(os_, lambda k2: galerkin.helmholtz_matrix(mats, a, b, k2))
    _check_solve(got, ref, fo, systems, sizes[0] - 2, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", [(["biharmonic"], [40]), (["biharmonic", "r2c"], [34, 18]),
                                          (["biharmonic", "c2c", "r2c"], [32, 33, 34]),
                                          (["biharmonic", "c2c"], [67, 9]),
                                          (["biharmonic", "c2c", "r2c"], [32, 16, 16]),
                                          (["biharmonic", "c2c", "r2c"], [20, 9, 9])])
@pytest.mark.parametrize("a,b,c", [(1.0, 0.0, 0.0), (1.3, -0.4, 2.0), (0.0, 0.0, 1.0), (0.0, 1.0, -5.0)])
def test_biharmonic_solve(kinds, sizes, prec, a, b, c):
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("poisson2d", 12)
    f = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        f = f + 1j * g.standard_normal(gs.spectral_shape)
    f[sizes[0] - 4:] = 0
    fd = to_dev(f, gs.spectral_dtype)
    fo = to_np(fd)
    got = to_np(gs.biharmonic_solve(a, b, c, fd))
    ref = os_.biharmonic(a, b, c, fo)
    mats = os_.matrices()
    systems = _column_systems(os_, lambda k2: galerkin.biharmonic_matrix(mats, a, b, c, k2))
    _check_solve(got, ref, fo, systems, sizes[0] - 4, prec)


def _check_solve(got, ref, f, systems, nb, prec):
    assert np.all(got[nb:] == 0)
    if prec == "f32":
        assert rel(got, ref) < 2e-6
        return
    cond = max(np.linalg.cond(M) for M in systems)
    assert rel(got, ref) < max(1e-12, 32 * EPS * cond), (rel(got, ref), cond)
    G = got.reshape(got.shape[0], -1)
    F = f.reshape(f.shape[0], -1)
    for j, M in enumerate(systems):
        x = G[:nb, j]
        r = np.linalg.norm(M @ x - F[:nb, j])
        denom = np.linalg.norm(M, 2) * np.linalg.norm(x) + np.linalg.norm(F[:nb, j])
        assert r <= 16 * EPS * denom, (j, r / denom)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_poisson2d_manufactured(prec, tol):
    N = (32, 32)
    kinds = ["dirichlet", "r2c"]
    gs = gspace(kinds, N, prec)
    x, y = inputs.mesh(kinds, N)
    fd = to_dev(inputs.poisson2d_f(x, y), gs.physical_dtype)
    u = to_np(gs.helmholtz(-1.0, 0.0, fd))
    assert rel(u, inputs.poisson2d_u(x, y)) < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("size", [12, 64])
def test_box3d_manufactured(prec, tol, size):
    N = (size, size, size)
    for kind in ("dirichlet", "biharmonic"):
        kinds = [kind, "c2c", "r2c"]
        gs = gspace(kinds, N, prec)
        x, y, z = inputs.mesh(kinds, N)
        if kind == "dirichlet":
            fd = to_dev(np.broadcast_to(inputs.box3d_f_poisson(x, y, z), N), gs.physical_dtype)
            u = to_np(gs.helmholtz(-1.0, 0.0, fd))
        else:
            fd = to_dev(np.broadcast_to(inputs.box3d_f_biharmonic(x, y, z), N), gs.physical_dtype)
            u = to_np(gs.biharmonic(1.0, 0.0, 0.0, fd))
        assert rel(u, np.broadcast_to(inputs.box3d_u(x, y, z), N)) < tol, kind


def test_errors_are_raised():
    from paper_1708_03188_gb300.sgm import SgmError
    gs = gspace(["dirichlet", "r2c"], [16, 16], "f32")
    x = gs.empty_physical()
    with pytest.raises(ValueError):
        gs.forward(torch.zeros(3, device="cuda"))
    y = gs.empty_spectral()
    with pytest.raises(SgmError):
        gs.helmholtz_solve(0.0, 0.0, y)           # singular
    gb = gspace(["biharmonic", "r2c"], [16, 16], "f32")
    with pytest.raises(SgmError):
        gb.helmholtz_solve(1.0, 0.0, gb.empty_spectral())   # wrong basis
    with pytest.raises(SgmError):
        gs.helmholtz(-1.0, 0.0, x, out=x)           # aliasing physical in/out


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 5e-5)])
@pytest.mark.parametrize("N", [4096, 4093])
def test_dirichlet_at_the_size_limit_manufactured(prec, tol, N):
    # the largest Chebyshev axis (4096) and a large prime one (4093, generic-radix DFT), 1-D and
    # 2-D: u = (1 - x^2) exp(x) sin(3x) (times cos 2y in 2-D) against a u'' - alpha u = f with
    # f in closed form
    def exact(x):
        return (1 - x * x) * np.exp(x) * np.sin(3 * x)

    def second(x):
        e, s3, c3 = np.exp(x), np.sin(3 * x), np.cos(3 * x)
        g, g1, g2 = 1 - x * x, -2 * x, -2.0
        h, h1, h2 = e * s3, e * (s3 + 3 * c3), e * (-8 * s3 + 6 * c3)
        return g2 * h + 2 * g1 * h1 + g * h2

    alpha = 40.0
    x = inputs.cheb_points(N)
    gs = gspace(["dirichlet"], [N], prec)
    u = to_np(gs.helmholtz(1.0, -alpha, to_dev(second(x) - alpha * exact(x), gs.physical_dtype)))
    assert rel(u, exact(x)) < tol
    # 2-D: lap u - alpha u with u = exact(x) cos 2y, so f = (u_xx - (4 + alpha) u) cos 2y
    g2 = gspace(["dirichlet", "r2c"], [N, 8], prec)
    xx, yy = inputs.mesh(["dirichlet", "r2c"], (N, 8))
    f2 = (second(xx) - (4.0 + alpha) * exact(xx)) * np.cos(2 * yy)
    u2 = to_np(g2.helmholtz(1.0, -alpha, to_dev(f2, g2.physical_dtype)))
    assert rel(u2, exact(xx) * np.cos(2 * yy)) < tol
