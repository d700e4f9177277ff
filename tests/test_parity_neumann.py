"""GPU parity of the Shen Neumann basis (Sec. 3.1 ShenNeumannBasis, phi_k = T_k - (k/(k+2))^2 T_{k+2})
against the FP64 oracle: transforms, the Helmholtz solve (with the singular constant column of a
Poisson problem, read as u_hat_0 = 0 with the phi_0 equation dropped), the physical-to-physical
solve (the one-tile and the streaming pipelines) and projected derivatives.

Tolerances as in test_parity_space.py: f64 1e-12 (transforms, well-conditioned solves), f32 4e-6
(transforms), 2e-6 (FP64 solves of FP32 data); projected derivatives f64 1e-12, f32 2^-22.
"""
import numpy as np
import pytest
import torch

from oracle import quadrature
from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu


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


SPACES = [(["neumann"], [33]), (["neumann"], [64]), (["neumann", "r2c"], [32, 18]),
          (["neumann", "c2c", "r2c"], [24, 8, 12]), (["neumann", "c2c", "r2c"], [64, 32, 32])]
TOL_T = {"f64": 1e-12, "f32": 4e-6}
TOL_S = {"f64": 1e-11, "f32": 2e-6}


def physical(sp, item):
    g = inputs.rng("box3d", 800 + item)
    x = g.standard_normal(sp.physical_shape)
    if not sp.real_physical:
        x = x + 1j * g.standard_normal(sp.physical_shape)
    return x


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", SPACES)
def test_neumann_transforms(kinds, sizes, prec):
    sp = gspace(kinds, sizes, prec)
    osp = OSpace(kinds, sizes)
    ud = to_dev(physical(sp, len(sizes)), sp.physical_dtype)
    u = to_np(ud)
    S = sp.scalar_product(ud)
    assert rel(to_np(S), osp.scalar_product(u)) < TOL_T[prec]
    F = sp.forward(ud)
    ref = osp.forward(u)
    assert rel(to_np(F), ref) < TOL_S[prec]
    B = sp.backward(to_dev(ref, sp.spectral_dtype))
    assert rel(to_np(B), osp.backward(to_np(to_dev(ref, sp.spectral_dtype)))) < TOL_T[prec]
    sp.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", SPACES)
@pytest.mark.parametrize("a,b", [(-1.0, 0.0), (1.0, -50.0), (1.0, 4.0)])
def test_neumann_helmholtz_solve(kinds, sizes, prec, a, b):
    # (-1, 0): Poisson, singular in the constant Fourier column; (1, 4): singular where kappa2 = 4
    sp = gspace(kinds, sizes, prec)
    osp = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 830 + len(sizes))
    f = g.standard_normal(sp.spectral_shape)
    if not sp.real_spectral:
        f = f + 1j * g.standard_normal(sp.spectral_shape)
    f[sizes[0] - 2:] = 0
    fd = to_dev(f, sp.spectral_dtype)
    got = to_np(sp.helmholtz_solve(a, b, fd))
    ref = osp.helmholtz(a, b, to_np(fd))
    assert rel(got, ref) < TOL_S[prec], rel(got, ref)
    sp.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("sizes", [[32, 16], [64, 32]])
def test_neumann_poisson_manufactured(sizes, prec, tol):
    # -lap u = f, u = cos(pi x) sin(2y): u'(+-1) = 0, every excited column has kappa2 = 4
    sp = gspace(["neumann", "r2c"], sizes, prec)
    x, y = inputs.mesh(sp.kinds, sizes)
    u = np.cos(np.pi * x) * np.sin(2 * y)
    f = (np.pi ** 2 + 4) * u
    got = to_np(sp.helmholtz(-1.0, 0.0, to_dev(np.broadcast_to(f, sizes), sp.physical_dtype)))
    assert rel(got, np.broadcast_to(u, sizes)) < tol
    sp.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_neumann_fused_solve_3d_against_oracle(prec, tol):
    # the physical-to-physical Helmholtz solve (the streaming pipeline on FP32) against the oracle's
    # scalar product, dense LU and backward sum on the same random right-hand side
    kinds, sizes = ["neumann", "c2c", "r2c"], [64, 32, 64]
    sp = gspace(kinds, sizes, prec)
    osp = OSpace(kinds, sizes)
    fd = to_dev(physical(sp, 9), sp.physical_dtype)
    got = to_np(sp.helmholtz(1.0, -30.0, fd))
    ref = osp.backward(osp.helmholtz(1.0, -30.0, osp.scalar_product(to_np(fd))))
    assert rel(got, ref) < tol, rel(got, ref)
    sp.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2.0 ** -22)])
def test_neumann_project_dx(prec, tol):
    kinds, sizes = ["neumann", "c2c"], [20, 6]
    sp = gspace(kinds, sizes, prec)
    osp = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 850)
    uh = g.standard_normal(sp.spectral_shape) + 1j * g.standard_normal(sp.spectral_shape)
    ud = to_dev(uh, sp.spectral_dtype)
    for axis, m in ((0, 1), (0, 2), (1, 1)):
        assert rel(to_np(sp.project_dx(ud, axis, m)), osp.project_dx(to_np(ud), axis, m)) < tol
    sp.close()
