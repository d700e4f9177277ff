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
- Backward transform of a full random spectrum (complex N(0,1) exp(-|k|/16) on the basis rows,
  Hermitian on the two self-conjugate R2C planes) on sampled output rows u(x_j, y_i, :): the
  oracle's basis values summed over k, a dense inverse DFT over l1 and the Hermitian sum over l2.
  FP32 1e-5 and FP64 1e-12 per row, relative to the field's root-mean-square row.
- The fused physical-to-physical path the bench times (sgm_helmholtz / sgm_biharmonic, FP64
  spectral intermediate) on a right-hand side with 24 Fourier modes of white-noise x-profiles,
  over the whole box: the oracle solves each mode's column (quadrature scalar product, dense
  LU with its kappa^2, basis sum) and the exact output is the sum of the 24 rank-one fields.
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


def hermitian_planes(c, M1):
    """Make the l2 = 0 and l2 = M2/2 planes Hermitian in l1 (c(-l1) = conj c(l1)), so that every
    reading of the C2R backward gives the same real field."""
    for l2 in (0, c.shape[2] - 1):
        plane = c[:, :, l2]
        neg = (-np.arange(M1)) % M1
        plane[:] = 0.5 * (plane + np.conj(plane[:, neg]))
    return c


def oracle_row(kind, c, j, i):
    """u(x_j, y_i, z) for all z from the spectral array c (N, M1, M2/2 + 1) by dense sums."""
    n0, M1, H = c.shape
    x, _ = quadrature.points(kind, n0)
    phi = quadrature.basis_values(kind, n0, x[j:j + 1])[0]            # phi_k(x_j), k < nb
    a = np.tensordot(phi, c[:phi.shape[0]], axes=(0, 0))              # (M1, H)
    yi = 2 * np.pi * i / M1
    g = np.exp(1j * fourier.wavenumbers(M1) * yi) @ a                  # (H,)
    M2 = 2 * (H - 1)
    z = 2 * np.pi * np.arange(M2) / M2
    w = np.full(H, 2.0)
    w[0] = w[-1] = 1.0
    return np.real(np.exp(1j * np.outer(z, fourier.wavenumbers(M2, r2c=True))) @ (w * g))


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f64", 1e-12)])
@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_backward_random_spectrum_sampled_rows(kind, prec, tol):
    from paper_1708_03188_gb300.sgm import Space
    sp = Space([kind, "c2c", "r2c"], SHAPE, precision=prec)
    nb = N - (2 if kind == "dirichlet" else 4)
    c = inputs.coefficients(sp.kinds, SHAPE, 16.0, item=720 + (kind == "biharmonic"), nvalid0=nb)
    c = hermitian_planes(np.ascontiguousarray(c), N)
    u = sp.backward(torch.from_numpy(c).to(sp.spectral_dtype).cuda()).cpu().numpy().astype(np.float64)
    g = inputs.rng("box3d", 730)
    rows = [(0, 0), (N - 1, N - 1), (N // 2, 1)] + list(zip(g.integers(0, N, 13).tolist(), g.integers(0, N, 13).tolist()))
    # Error of a row relative to the root-mean-square row of the field: near x = +-1 the basis
    # functions vanish (to second order for the biharmonic basis), so a row there is small
    # while the transform's rounding is set by the whole spectrum.
    scale = np.linalg.norm(u) / np.sqrt(u.shape[0] * u.shape[1])
    worst = 0.0
    for j, i in rows:
        e = np.linalg.norm(u[j, i] - oracle_row(kind, c, j, i)) / scale
        worst = max(worst, e)
        assert e < tol, (j, i, e)
    print(f"{kind} {prec} backward, {len(rows)} sampled rows: worst {worst:.2e}")
    sp.close()


@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_fused_solve_sparse_spectrum_full_box(kind):
    sp = gspace(kind)
    g = inputs.rng("box3d", 740 + (kind == "biharmonic"))
    x, wq = quadrature.points(kind, N)
    phi = quadrature.basis_values(kind, N, x)                          # (N, nb)
    y = 2 * np.pi * np.arange(N) / N
    k1 = fourier.wavenumbers(N)
    modes = [(0, 1), (1, 1), (128, 3), (129, 127), (255, 64), (64, 2)]  # FFT-order indices (i1, i2)
    modes += list(zip(g.integers(0, N, 18).tolist(), g.integers(1, N // 2, 18).tolist()))
    modes = list(dict.fromkeys(modes))
    f = np.zeros(SHAPE)
    exact = np.zeros(SHAPE)
    for i1, i2 in modes:
        h = g.standard_normal(N) + 1j * g.standard_normal(N)            # x-profile at the Gauss points
        ey = np.exp(1j * k1[i1] * y)
        ez = np.exp(1j * i2 * y)
        f += np.real(h[:, None, None] * ey[None, :, None] * ez[None, None, :])
        S = (phi * wq[:, None]).T @ (0.5 * h)                           # column (i1, i2) coefficient h/2
        rhs = np.zeros(N, complex)
        rhs[:phi.shape[1]] = S
        uh = column_solve(kind, rhs, k1[i1] ** 2 + i2 ** 2)
        v = 2.0 * (phi @ uh[:phi.shape[1]])                             # C2R doubles l2 > 0
        exact += np.real(v[:, None, None] * ey[None, :, None] * ez[None, None, :])
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    u = sp.helmholtz(-1.0, 0.0, fd) if kind == "dirichlet" else sp.biharmonic(1.0, 0.0, 0.0, fd)
    ex = torch.from_numpy(exact).cuda()
    err = float(torch.linalg.vector_norm(u.double() - ex) / torch.linalg.vector_norm(ex))
    print(f"{kind} fused 256^3 solve, {len(modes)} random modes: {err:.2e}")
    assert err < 1e-5
    sp.close()
