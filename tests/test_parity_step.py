"""GPU parity at the size of the timed step: the 256^3 FP32 Poisson and biharmonic boxes
(Shen-Dirichlet / Shen-biharmonic x C2C 256 x R2C 256), through the same calls bench.py times.

- Physical-to-physical solves of the manufactured u = (1-x^2)^2 sin y cos 2z over the whole array.
  Measured relative L2 errors are 1.6e-7 (Poisson) and 1.0e-7 (biharmonic); the tolerance is the
  2e-5 of the smaller FP32 manufactured cases.
- Scalar product of white noise, and the spectral solves, on sampled columns against the oracle
  computed column by column: a dense 2-D DFT sum for the column's Fourier coefficient at every
  x_j, the quadrature scalar product along x, and a dense LU of the column's Galerkin system with
  its own kappa^2.  Tolerance 1e-5 relative per column (FP32 transforms: ~log2(N) 2^-24 per pass,
  three passes; FP64 eliminations, rounded to FP32 once).
"""
import numpy as np
import pytest
import torch

from oracle import fourier, galerkin, quadrature
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
N = 256
SHAPE = (N, N, N)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def gspace(kind):
    from paper_1708_03188_gb300.sgm import Space
    return Space([kind, "c2c", "r2c"], SHAPE, precision="f32")


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def column_scalar_product(kind, u, i1, i2):
    """S(F(u)) at Fourier column (i1, i2): dense DFT sums over y and z, then quadrature along x."""
    M1, M2 = u.shape[1], u.shape[2]
    y = 2 * np.pi * np.arange(M1) / M1
    z = 2 * np.pi * np.arange(M2) / M2
    l1 = fourier.wavenumbers(M1)[i1]
    l2 = fourier.wavenumbers(M2, r2c=True)[i2]
    phase = (l1 * y[:, None] + l2 * z[None, :])
    g = (np.tensordot(u, np.cos(phase), axes=([1, 2], [0, 1]))
         - 1j * np.tensordot(u, np.sin(phase), axes=([1, 2], [0, 1]))) / (M1 * M2)
    x, w = quadrature.points(kind, u.shape[0])
    phi = quadrature.basis_values(kind, u.shape[0], x)
    out = np.zeros(u.shape[0], complex)
    out[:phi.shape[1]] = (phi * w[:, None]).T @ g
    return out


def column_solve(kind, rhs, kappa2):
    mats = galerkin.matrices(kind, N)
    if kind == "dirichlet":
        system = lambda k2: galerkin.helmholtz_matrix(mats, -1.0, 0.0, k2)
    else:
        system = lambda k2: galerkin.biharmonic_matrix(mats, 1.0, 0.0, 0.0, k2)
    return galerkin.solve_columns(kind, N, rhs[:, None], np.array([kappa2]), system)[:, 0]


@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_step_manufactured_full_box(kind):
    sp = gspace(kind)
    x, y, z = inputs.mesh(sp.kinds, SHAPE)
    f = inputs.box3d_f_poisson(x, y, z) if kind == "dirichlet" else inputs.box3d_f_biharmonic(x, y, z)
    fd = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(f, SHAPE), dtype=np.float32)).cuda()
    u = sp.helmholtz(-1.0, 0.0, fd) if kind == "dirichlet" else sp.biharmonic(1.0, 0.0, 0.0, fd)
    exact = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(inputs.box3d_u(x, y, z), SHAPE))).cuda()
    err = float(torch.linalg.vector_norm(u.double() - exact) / torch.linalg.vector_norm(exact))
    print(f"{kind} 256^3 manufactured: {err:.2e}")
    assert err < 2e-5
    sp.close()


@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_step_sampled_columns(kind):
    sp = gspace(kind)
    g = inputs.rng("box3d", 700 + (kind == "biharmonic"))
    u = g.standard_normal(SHAPE).astype(np.float32)
    S = sp.scalar_product(torch.from_numpy(u).cuda())
    U = sp.helmholtz_solve(-1.0, 0.0, S) if kind == "dirichlet" else sp.biharmonic_solve(1.0, 0.0, 0.0, S)
    torch.cuda.synchronize()
    spec = sp.spectral_shape
    cols = [(0, 0), (1, 0), (0, 1), (N // 2, N // 2), (N - 1, 3)]
    cols += list(zip(g.integers(0, spec[1], 19).tolist(), g.integers(0, spec[2], 19).tolist()))
    k1 = fourier.wavenumbers(N)
    k2 = fourier.wavenumbers(N, r2c=True)
    u64 = u.astype(np.float64)
    for i1, i2 in cols:
        s_gpu = S[:, i1, i2].cpu().numpy().astype(np.complex128)
        e_s = rel(s_gpu, column_scalar_product(kind, u64, i1, i2))
        assert e_s < 1e-5, ("scalar product", i1, i2, e_s)
        e_u = rel(U[:, i1, i2].cpu().numpy().astype(np.complex128),
                  column_solve(kind, s_gpu, k1[i1] ** 2 + k2[i2] ** 2))
        assert e_u < 1e-5, ("solve", i1, i2, e_u)
    sp.close()
