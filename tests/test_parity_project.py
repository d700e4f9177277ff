"""GPU parity: projected derivatives project(Dx(u, axis, m), W0) (Sec. 5) against the FP64 oracle.

Tolerances (relative L2 over the array):
  f64   1e-12   plain FP64 recurrence; its rounding stays near sqrt(N) * 2^-53 of the output
  f32   2^-22   every intermediate is a float pair (~2^-44); the output is rounded to FP32
                once (<= 2^-24 per element, ~2^-25 relative L2 in practice)
The oracle receives exactly the values the GPU received.  Rows of u_hat past the basis size
hold random values, which both sides must ignore.
"""
import numpy as np
import pytest
import torch

from oracle import fourier
from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 2.0 ** -22}


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
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def random_coefficients(gs, item):
    g = inputs.rng("box3d", 500 + item)
    x = g.standard_normal(gs.spectral_shape)
    if not gs.real_spectral:
        x = x + 1j * g.standard_normal(gs.spectral_shape)
    return x


SPACES = [
    (["chebyshev"], [2], None),                       # smallest bases
    (["chebyshev"], [7], None),
    (["dirichlet"], [4], None),
    (["biharmonic"], [6], None),
    (["dirichlet"], [201], None),                     # odd N, many register chunks per thread
    (["biharmonic"], [64], None),
    (["biharmonic", "r2c"], [33, 30], None),
    (["chebyshev", "c2c"], [17, 9], None),
    (["dirichlet", "c2c", "r2c"], [24, 10, 18], None),
    (["biharmonic", "c2c", "r2c"], [40, 6, 301], None),  # 906 columns: 8 CTAs, the last one ragged
    (["dirichlet", "c2c"], [16, 12], [(-1.0, 1.0), (0.0, 7.0)]),
    (["legendre"], [9], None),                        # Legendre bases: W0 is the regular Legendre basis
    (["legendre_dirichlet"], [41], None),
    (["legendre_biharmonic", "r2c"], [13, 6], None),
    (["legendre_biharmonic", "c2c", "r2c"], [40, 6, 301], None),
    (["c2c", "r2c"], [12, 16], None),                 # Fourier-only spaces: one row, W0 = the space
    (["c2c"], [30], None),
    (["c2c", "c2c"], [16, 16], [(-50.0, 50.0), (-50.0, 50.0)]),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes,domain", SPACES, ids=lambda v: "-".join(map(str, v)) if v else "default")
def test_project_dx(kinds, sizes, domain, prec):
    gs = gspace(kinds, sizes, prec, domain)
    os_ = OSpace(kinds, sizes, domains=domain)
    x = random_coefficients(gs, len(kinds) * 100 + sizes[0])
    xd = to_dev(x, gs.spectral_dtype)
    xo = to_np(xd)
    worst = 0.0
    for axis in range(len(kinds)):
        for m in range(5):
            got = to_np(gs.project_dx(xd, axis, m))
            e = rel(got, os_.project_dx(xo, axis, m))
            worst = max(worst, e)
            assert e < TOL[prec], (axis, m, e)
    print(f"project_dx {kinds} {sizes} {prec}: worst {worst:.2e}")


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-3)])
def test_project_dx_box3d_derivative_of_the_solution(prec, tol):
    """The example of Sec. 5: du/dx of u = (1-x^2)^2 sin y cos 2z, given on the biharmonic space,
    projected onto the regular Chebyshev space and evaluated there by its backward transform.

    The derivative amplifies the forward transform's rounding in high modes: with noise of one
    unit roundoff u in every coefficient, the oracle gives a relative error of ~1400 u at N = 48
    (about 0.6 N^2).  FP32 transforms carry up to ~log2(N) u, hence 1e-3 (FP32) and 1e-11 (FP64)."""
    N = (48, 16, 16)
    kinds = ["biharmonic", "c2c", "r2c"]
    gs = gspace(kinds, N, prec)
    w0 = gs.chebyshev_space()
    x, y, z = inputs.mesh(kinds, N)
    u = np.broadcast_to(inputs.box3d_u(x, y, z), N)
    u_hat = gs.forward(to_dev(u, gs.physical_dtype))
    du = to_np(w0.backward(gs.project_dx(u_hat, 0, 1)))
    exact = np.broadcast_to(-4 * x * (1 - x ** 2) * np.sin(y) * np.cos(2 * z), N)
    assert rel(du, exact) < tol
    d2z = to_np(w0.backward(gs.project_dx(u_hat, 2, 2)))
    assert rel(d2z, -4 * u) < tol


@pytest.mark.parametrize("axis,m", [(0, 1), (0, 4), (1, 1), (2, 2)])
def test_project_dx_full_box_sampled(axis, m):
    """256^3 FP32 biharmonic x C2C x R2C box (the size of the timed workload), one launch over
    all 33,024 columns, checked on 48 sampled columns against the oracle column by column."""
    N = 256
    gs = gspace(["biharmonic", "c2c", "r2c"], (N, N, N), "f32")
    g = inputs.rng("box3d", 600 + 10 * axis + m)
    shp = gs.spectral_shape
    gen = torch.Generator().manual_seed(int(g.integers(1 << 30)))
    xd = torch.view_as_complex(torch.randn(shp + (2,), generator=gen)).cuda()
    out = gs.project_dx(xd, axis, m)
    torch.cuda.synchronize()
    col1d = OSpace(["biharmonic"], [N])
    i1s = g.integers(0, shp[1], 48)
    i2s = g.integers(0, shp[2], 48)
    k1 = fourier.wavenumbers(N)
    k2 = fourier.wavenumbers(N, r2c=True)
    for i1, i2 in zip(i1s, i2s):
        col = xd[:, i1, i2].cpu().numpy().astype(np.complex128)
        if axis == 0:
            ref = col1d.project_dx(col, 0, m)
        else:
            k = k1[i1] if axis == 1 else k2[i2]
            ref = col1d.project_dx(col, 0, 0) * (1j * k) ** m
        got = out[:, i1, i2].cpu().numpy().astype(np.complex128)
        assert rel(got, ref) < TOL["f32"], (i1, i2)


def test_project_dx_errors():
    from paper_1708_03188_gb300.sgm import SgmError
    gs = gspace(["dirichlet", "c2c"], (16, 8), "f64")
    x = torch.zeros(gs.spectral_shape, dtype=gs.spectral_dtype, device="cuda")
    for axis, m in ((2, 1), (-1, 1), (0, 5), (1, -1)):
        with pytest.raises(SgmError):
            gs.project_dx(x, axis, m)
    with pytest.raises(SgmError):
        gs.project_dx(x, 0, 1, out=x)                 # in place is refused
    w0 = gs.chebyshev_space()
    assert w0.kinds == ("chebyshev", "c2c") and w0.spectral_shape == gs.spectral_shape


# ---- projection onto a Shen space: sgm_project (Sec. 5 project with a composite target) -----------
PROJECT_CASES = [
    (["dirichlet"], [16], "biharmonic"),
    (["biharmonic"], [33], "dirichlet"),
    (["chebyshev"], [24], "dirichlet"),
    (["chebyshev", "r2c"], [24, 16], "biharmonic"),
    (["dirichlet", "c2c", "r2c"], [20, 8, 12], "dirichlet"),
    (["biharmonic", "c2c", "r2c"], [40, 6, 10], "dirichlet"),
    (["dirichlet", "c2c"], [64, 5], "biharmonic"),
    (["legendre_dirichlet", "r2c"], [18, 8], "legendre_biharmonic"),
    (["legendre_biharmonic", "c2c", "r2c"], [22, 4, 6], "legendre_dirichlet"),
]
# FP32: the derivative's regular coefficients are rounded to FP32 once before the (FP64)
# Galerkin projection, whose coefficient-space condition grows with the target's mass matrix
PROJECT_TOL = {"f64": 1e-11, "f32": 2.0 ** -18}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes,target", PROJECT_CASES)
def test_project_onto_shen_space(kinds, sizes, target, prec):
    sp = gspace(kinds, sizes, prec)
    tk = [target] + list(kinds[1:])
    tg = gspace(tk, sizes, prec)
    osp = OSpace(kinds, sizes)
    uh = random_coefficients(sp, 60 + len(sizes))
    ud = to_dev(uh, sp.spectral_dtype)
    uh_used = to_np(ud)
    worst = 0.0
    for axis in range(len(kinds)):
        for m in (0, 1, 2):
            got = to_np(sp.project(ud, axis, m, tg))
            ref = osp.project_dx(uh_used, axis, m, target=target)
            e = rel(got, ref)
            worst = max(worst, e)
            assert e < PROJECT_TOL[prec], (axis, m, e)
            nt = sizes[0] - (2 if "dirichlet" in target else 4)
            assert np.all(got[nt:] == 0)
    print(f"project {kinds} {sizes} -> {target} {prec}: worst {worst:.2e}")
    sp.close()
    tg.close()


def test_project_rejects_mismatched_targets():
    from paper_1708_03188_gb300.sgm import SgmError
    sp = gspace(["dirichlet", "c2c"], [16, 8], "f64")
    u = sp.empty_spectral().zero_()
    for kinds, sizes, prec in ((["biharmonic", "c2c"], [16, 9], "f64"), (["biharmonic", "c2c"], [16, 8], "f32"),
                               (["legendre_biharmonic", "c2c"], [16, 8], "f64"), (["biharmonic", "r2c"], [16, 14], "f64")):
        tg = gspace(kinds, sizes, prec)
        out = tg.empty_spectral()
        with pytest.raises((SgmError, ValueError)):
            from paper_1708_03188_gb300 import sgm
            sgm.check(sgm.lib().sgm_project(sp._h, 0, 1, sgm._ptr(u), tg._h, sgm._ptr(out), sgm._stream(None)))
        tg.close()
    sp.close()
