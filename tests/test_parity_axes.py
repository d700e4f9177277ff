"""GPU parity of spaces in another axis order (the axes option of Sec. 4: the Dirichlet basis
along the second axis, TensorProductSpace((K1, K0), axes=(1, 0))).  Such a space is by definition
the canonical one (polynomial axis first, R2C axis last) with its arrays' axes permuted, so the
oracle computes on the canonical space and its results are transposed to the array order; the
paper's 2-D Poisson example with the axes flipped is also checked against its closed form.
Tolerances as in test_parity_space.py (f64 1e-12 transforms, 1e-11 solves; f32 4e-6 / 2e-6).
"""
import numpy as np
import pytest
import torch

from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
POLY = ("chebyshev", "dirichlet", "biharmonic", "neumann", "legendre", "legendre_dirichlet", "legendre_biharmonic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def canonical_order(kinds):
    return ([d for d, k in enumerate(kinds) if k in POLY] + [d for d, k in enumerate(kinds) if k == "c2c"]
            + [d for d, k in enumerate(kinds) if k == "r2c"])


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


CASES = [(["r2c", "dirichlet"], [33, 32]), (["c2c", "biharmonic", "r2c"], [8, 20, 12]),
         (["r2c", "c2c", "neumann"], [12, 8, 16]), (["c2c", "dirichlet"], [10, 16]),
         (["c2c", "r2c", "chebyshev"], [6, 10, 9])]
TOL_T = {"f64": 1e-12, "f32": 4e-6}
TOL_S = {"f64": 1e-11, "f32": 2e-6}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", CASES)
def test_permuted_space_against_transposed_oracle(kinds, sizes, prec):
    from paper_1708_03188_gb300.sgm import Space
    order = canonical_order(kinds)
    back = np.argsort(order)
    sp = Space(kinds, sizes, precision=prec)
    osp = OSpace([kinds[o] for o in order], [sizes[o] for o in order])
    to_c = lambda a: np.transpose(a, order)           # array order -> canonical
    to_a = lambda c: np.transpose(c, back)            # canonical -> array order
    g = inputs.rng("box3d", 880 + len(sizes))
    u = g.standard_normal(sp.physical_shape)
    if not sp.real_physical:
        u = u + 1j * g.standard_normal(sp.physical_shape)
    ud = to_dev(u, sp.physical_dtype)
    uo = to_c(to_np(ud))
    assert rel(to_np(sp.scalar_product(ud)), to_a(osp.scalar_product(uo))) < TOL_T[prec]
    uh_ref = osp.forward(uo)
    assert rel(to_np(sp.forward(ud)), to_a(uh_ref)) < TOL_S[prec]
    uhd = to_dev(to_a(uh_ref), sp.spectral_dtype)
    assert rel(to_np(sp.backward(uhd)), to_a(osp.backward(to_c(to_np(uhd))))) < TOL_T[prec]
    pk = next(k for k in kinds if k in POLY)
    if pk in ("dirichlet", "neumann"):
        got = to_np(sp.helmholtz_solve(1.0, -20.0, sp.scalar_product(ud)))
        ref = to_a(osp.helmholtz(1.0, -20.0, osp.scalar_product(uo)))
        assert rel(got, ref) < TOL_S[prec]
        got = to_np(sp.helmholtz(1.0, -20.0, ud))
        assert rel(got, to_a(osp.backward(osp.helmholtz(1.0, -20.0, osp.scalar_product(uo))))) < TOL_S[prec]
    elif pk == "biharmonic":
        got = to_np(sp.biharmonic(1.0, 0.0, 3.0, ud))
        assert rel(got, to_a(osp.backward(osp.biharmonic(1.0, 0.0, 3.0, osp.scalar_product(uo))))) < 1e-5
    for axis in range(len(kinds)):
        got = to_np(sp.project_dx(uhd, axis, 1))
        ref = to_a(osp.project_dx(to_c(to_np(uhd)), int(back[axis]), 1))
        assert rel(got, ref) < (1e-12 if prec == "f64" else 2.0 ** -22), axis
    sp.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_poisson_2d_with_flipped_axes(prec, tol):
    # Sec. 4 with the Fourier basis first: u(y, x) = sin(pi x)(1 + cos 2y + sin 3y) on
    # [0, 2 pi) x [-1, 1], -lap u = f, arrays indexed [y, x]
    from paper_1708_03188_gb300.sgm import Space
    sizes = [33, 32]
    sp = Space(["r2c", "dirichlet"], sizes, precision=prec)
    y = 2 * np.pi * np.arange(sizes[0]) / sizes[0]
    x = inputs.cheb_points(sizes[1])
    u = (1 + np.cos(2 * y) + np.sin(3 * y))[:, None] * np.sin(np.pi * x)[None, :]
    f = inputs.poisson2d_f(x[None, :], y[:, None]) * np.ones(sizes)
    got = to_np(sp.helmholtz(-1.0, 0.0, to_dev(f, sp.physical_dtype)))
    assert rel(got, u) < tol
    sp.close()
