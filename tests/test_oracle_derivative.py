"""Pins for the oracle's projected derivative, project(Dx(u, axis, m), W0) of Sec. 5 (CPU only).

The oracle builds the projection from quadrature Galerkin matrices.  These tests fix it with
routes that share none of that code:
  - exact Chebyshev coefficients of p^(m) for random integer polynomials p that satisfy the basis'
    boundary conditions, by the power rule on monomials and the identity
    x^n = 2^(1-n) sum'_j C(n, j) T_{n-2j} (the T_0 term halved), in exact rational arithmetic;
  - the closed-form coefficients of derivatives of u = (1 - x^2)^2 sin y cos 2z;
  - the physical derivative of a Fourier mode on a non-2pi domain at the mesh points;
  - composition (d/dx of d/dx is d^2/dx^2) and commutation of mixed derivatives.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from oracle import quadrature
from oracle.space import Space
from paper_1708_03188_gb300 import inputs


def poly_mul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def poly_der(p, m):
    for _ in range(m):
        p = [i * p[i] for i in range(1, len(p))] or [Fraction(0)]
    return p


def monomials_to_chebyshev(p, N):
    """Chebyshev coefficients (length N) of sum_n p[n] x^n, exactly."""
    c = [Fraction(0)] * max(N, len(p))
    for n, a in enumerate(p):
        if a == 0:
            continue
        if n == 0:
            c[0] += a
            continue
        for j in range(n // 2 + 1):
            t = Fraction(comb(n, j), 2 ** (n - 1))
            if n - 2 * j == 0:
                t /= 2
            c[n - 2 * j] += a * t
    return c[:N]


def poly_eval(p, x):
    out = np.zeros_like(x)
    for a in reversed(p):
        out = out * x + float(a)
    return out


@pytest.mark.parametrize("kind", ["chebyshev", "dirichlet", "biharmonic"])
@pytest.mark.parametrize("N", [8, 13])
def test_project_dx_exact_polynomials(kind, N):
    g = np.random.default_rng(17 + N)
    bc = {"chebyshev": 0, "dirichlet": 1, "biharmonic": 2}[kind]
    q = [Fraction(int(v)) for v in g.integers(-9, 10, N - 2 * bc)]
    p = q
    for _ in range(bc):                                   # (1 - x^2)^bc q(x), degree N - 1
        p = poly_mul(p, [Fraction(1), Fraction(0), Fraction(-1)])
    sp = Space([kind], [N])
    x, _ = quadrature.gauss_points(N)
    u_hat = sp.forward(poly_eval(p, x))
    for m in range(5):
        exact = np.array([float(v) for v in monomials_to_chebyshev(poly_der(p, m), N)])
        got = sp.project_dx(u_hat, 0, m)
        scale = max(np.max(np.abs(exact)), 1.0)
        assert np.max(np.abs(got - exact)) < 1e-12 * scale, (kind, N, m)


def test_project_dx_box3d_closed_forms():
    # u = (1-x^2)^2 sin y cos 2z; (1-x^2)^2 = 3/8 T_0 - 1/2 T_2 + 1/8 T_4, sin y -> -i/2 at l = 1 and
    # i/2 at l = -1, cos 2z -> 1/2 at R2C index 2.
    N = (12, 8, 8)
    for kind in ("dirichlet", "biharmonic"):
        sp = Space([kind, "c2c", "r2c"], N)
        x, y, z = inputs.mesh(sp.kinds, N)
        u_hat = sp.forward(np.broadcast_to(inputs.box3d_u(x, y, z), N))
        cheb_u = np.zeros(12)
        cheb_u[[0, 2, 4]] = [3 / 8, -1 / 2, 1 / 8]
        cheb_dx = np.zeros(12)
        cheb_dx[[1, 3]] = [-1.0, 1.0]                      # d/dx (1-x^2)^2 = -T_1 + T_3
        cheb_dxx = np.zeros(12)
        cheb_dxx[[0, 2]] = [2.0, 6.0]                      # -4 + 12 x^2 = 2 T_0 + 6 T_2

        def field(cheb, fy):                               # fy: coefficients at l = 1, -1
            out = np.zeros(sp.spectral_shape, complex)
            out[:, 1, 2] = cheb * fy[0] * 0.5
            out[:, -1, 2] = cheb * fy[1] * 0.5
            return out

        sin_y = (-0.5j, 0.5j)
        cos_y = (0.5, 0.5)
        cases = [
            (0, 0, field(cheb_u, sin_y)),
            (0, 1, field(cheb_dx, sin_y)),
            (0, 2, field(cheb_dxx, sin_y)),
            (0, 3, field(np.eye(12)[1] * 24.0, sin_y)),     # 24 x
            (0, 4, field(np.eye(12)[0] * 24.0, sin_y)),
            (1, 1, field(cheb_u, cos_y)),
            (1, 2, -field(cheb_u, sin_y)),
            (2, 1, field(cheb_u, (-0.5j * 2j, 0.5j * 2j))),  # -2 sin y sin 2z
            (2, 2, -4 * field(cheb_u, sin_y)),
        ]
        for axis, m, expect in cases:
            got = sp.project_dx(u_hat, axis, m)
            # the forward transform's roundoff in high modes grows ~N^2 per derivative
            assert np.max(np.abs(got - expect)) < 1e-13 * 10.0 ** m, (kind, axis, m)


def test_project_dx_fourier_domain_scaling():
    # d/dx of sin(2 pi 3 x / 100) on [-50, 50) x [-50, 50), evaluated at the mesh points
    M = 16
    sp = Space(["c2c", "r2c"], [M, M], domains=[(-50.0, 50.0), (-50.0, 50.0)])
    xs = -50.0 + 100.0 * np.arange(M) / M
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    k = 2 * np.pi / 100.0
    u = np.sin(3 * k * X) * np.cos(2 * k * Y)
    u_hat = sp.forward(u)
    du = sp.backward(sp.project_dx(u_hat, 0, 1))
    assert np.max(np.abs(du - 3 * k * np.cos(3 * k * X) * np.cos(2 * k * Y))) < 1e-13
    d2 = sp.backward(sp.project_dx(u_hat, 1, 2))
    assert np.max(np.abs(d2 + (2 * k) ** 2 * u)) < 1e-13


@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_project_dx_composes_and_commutes(kind):
    N = (14, 6, 8)
    sp = Space([kind, "c2c", "r2c"], N)
    w0 = Space(["chebyshev", "c2c", "r2c"], N)
    g = inputs.rng("box3d", 41)
    u = g.standard_normal(N)
    u_hat = sp.forward(u)
    two = sp.project_dx(u_hat, 0, 2)
    assert np.allclose(w0.project_dx(sp.project_dx(u_hat, 0, 1), 0, 1), two, rtol=0, atol=1e-11 * np.abs(two).max())
    xy = w0.project_dx(sp.project_dx(u_hat, 1, 1), 0, 1)
    yx = w0.project_dx(sp.project_dx(u_hat, 0, 1), 1, 1)
    assert np.allclose(xy, yx, rtol=0, atol=1e-12 * np.abs(xy).max())
    # the projection of u itself onto W0 represents the same function
    assert np.allclose(w0.backward(sp.project_dx(u_hat, 0, 0)), sp.backward(u_hat), rtol=0, atol=1e-13)


def test_project_dx_ignores_rows_past_the_basis():
    sp = Space(["biharmonic", "c2c"], [10, 4])
    g = inputs.rng("box3d", 42)
    u_hat = g.standard_normal((10, 4)) + 1j * g.standard_normal((10, 4))
    clean = u_hat.copy()
    clean[6:] = 0
    for axis, m in ((0, 1), (1, 1), (0, 0)):
        assert np.array_equal(sp.project_dx(u_hat, axis, m), sp.project_dx(clean, axis, m))


# ---- projection onto a Shen space (Sec. 5 project with a composite target basis) ---------------
def cheb_poly(k):
    """Monomial coefficients of T_k (three-term recurrence, exact)."""
    a, b = [Fraction(1)], [Fraction(0), Fraction(1)]
    if k == 0:
        return a
    for _ in range(k - 1):
        a, b = b, [x - y for x, y in zip([Fraction(0)] + [2 * v for v in b] + [Fraction(0)],
                                        a + [Fraction(0)] * 3)][:len(b) + 1]
    return b


def weighted_moment(n):
    """int_{-1}^{1} x^n (1 - x^2)^(-1/2) dx / pi = (n-1)!!/n!! for even n, 0 for odd n."""
    if n % 2:
        return Fraction(0)
    v = Fraction(1)
    for j in range(1, n, 2):
        v *= Fraction(j, j + 1)
    return v


def inner_w(p, q):
    """(p, q)_w / pi for monomial coefficient lists, exactly."""
    return sum(a * b * weighted_moment(i + j) for i, a in enumerate(p) for j, b in enumerate(q) if a and b)


def shen_poly(kind, k):
    """Monomial coefficients of the Chebyshev-family basis function psi_k of ``kind``."""
    P = quadrature.basis_coefficients(kind, k + 5)[k]
    out = [Fraction(0)] * (k + 5)
    for j, c in enumerate(P):
        if c:
            cf = Fraction(c).limit_denominator(1000)
            for i, t in enumerate(cheb_poly(j)):
                out[i] += cf * t
    return out


def solve_exact(A, b):
    """Gauss-Jordan elimination in Fractions."""
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("target", ["dirichlet", "biharmonic"])
@pytest.mark.parametrize("kind", ["chebyshev", "dirichlet", "biharmonic"])
def test_project_dx_onto_shen_space_exact_galerkin(kind, target):
    # The projection of p^(m) onto the Shen space W is the w-orthogonal (Galerkin) projection:
    # coefficients c with sum_j c_j (psi_j, psi_k)_w = (p^(m), psi_k)_w for every k.  Here every
    # inner product is an exact rational multiple of pi (Chebyshev-weight moments of monomials),
    # and the system is solved in Fractions: no quadrature, no NumPy series code.
    N = 10
    g = np.random.default_rng(31)
    bc = {"chebyshev": 0, "dirichlet": 1, "biharmonic": 2}[kind]
    q = [Fraction(int(v)) for v in g.integers(-9, 10, N - 2 * bc)]
    p = q
    for _ in range(bc):
        p = poly_mul(p, [Fraction(1), Fraction(0), Fraction(-1)])
    sp = Space([kind], [N])
    x, _ = quadrature.gauss_points(N)
    u_hat = sp.forward(poly_eval(p, x))
    nt = quadrature.num_basis(target, N)
    psi = [shen_poly(target, k) for k in range(nt)]
    B = [[inner_w(psi[j], psi[k]) for j in range(nt)] for k in range(nt)]
    for m in range(4):
        dp = poly_der(p, m)
        exact = solve_exact(B, [inner_w(dp, psi[k]) for k in range(nt)])
        exact = np.array([float(v) for v in exact] + [0.0] * (N - nt))
        got = sp.project_dx(u_hat, 0, m, target=target)
        scale = max(np.max(np.abs(exact)), 1.0)
        assert np.max(np.abs(got - exact)) < 1e-11 * scale, (kind, target, m)


def test_project_onto_shen_space_keeps_members():
    # a function already in W projects onto itself: biharmonic phi_l satisfy the Dirichlet
    # conditions, so their projection onto the Dirichlet space reproduces them exactly
    N = 12
    bs = Space(["biharmonic", "c2c"], [N, 4])
    ds = Space(["dirichlet", "c2c"], [N, 4])
    g = inputs.rng("box3d", 43)
    u_hat = np.zeros((N, 4), complex)
    u_hat[:N - 4] = g.standard_normal((N - 4, 4)) + 1j * g.standard_normal((N - 4, 4))
    w = bs.project_dx(u_hat, 0, 0, target="dirichlet")
    assert np.allclose(ds.backward(w), bs.backward(u_hat), rtol=0, atol=1e-13)
