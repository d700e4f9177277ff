"""Seeded synthetic inputs and manufactured solutions.

Shared by the tests, ``bench.py`` and ``smoke()``: it holds the sampling grids,
random number streams and closed-form manufactured functions, and none of the
method's transforms or solves.  Workload recipes (sizes and distributions of
the synthetic data):
  poisson2d      Dirichlet(32) x Fourier r2c(32) on [-1,1] x [0,2pi):
                 u = sin(pi x)(1 + cos 2y + sin 3y), f = -lap(u).
  box3d          Dirichlet or biharmonic(256) x Fourier c2c(256) x r2c(256):
                 u = (1-x^2)^2 sin y cos 2z; f = -lap(u) (Poisson) or lap^2(u).
  coefficients   complex N(0,1) * exp(-|k| / scale) on the valid spectral
                 indices, |k| the Euclidean norm of (l, m, n) with signed
                 Fourier wavenumbers.
  gl             u0 = 0.01 (N(0,1) + i N(0,1)) on an M x M periodic grid.
  batch1d        4096 problems, N = round(exp(U(ln 16, ln 2048))),
                 alpha ~ U(0, 1e4), f = sum_k c_k T_k with c_k ~ N(0,1) exp(-8k/N)
                 sampled at the Chebyshev-Gauss points.
Seeds: PCG64(1708031880 + 1000 * workload + item).
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

SEED_BASE = 1708031880
WORKLOADS = {"poisson2d": 0, "box3d": 1, "gl": 2, "batch": 3, "closure": 4}


def rng(workload, item=0):
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * WORKLOADS[workload] + item))


def cheb_points(N):
    """Chebyshev-Gauss sampling points cos((2j+1) pi / (2N))."""
    j = np.arange(N, dtype=np.float64)
    return np.cos((2 * j + 1) * np.pi / (2 * N))


def legendre_points(N):
    """Legendre-Gauss sampling points, descending like the Chebyshev points."""
    return np.polynomial.legendre.leggauss(N)[0][::-1].copy()


def fourier_points(M, domain=(0.0, 2 * np.pi)):
    a, b = domain
    return a + (b - a) * np.arange(M, dtype=np.float64) / M


def mesh(kinds, sizes, domains=None):
    """Broadcastable sampling grid, one array per axis (shape 1 except its own axis)."""
    out = []
    nd = len(sizes)
    for d, (k, n) in enumerate(zip(kinds, sizes)):
        if k in ("chebyshev", "dirichlet", "neumann", "biharmonic"):
            x = cheb_points(n)
        elif k in ("legendre", "legendre_dirichlet", "legendre_biharmonic"):
            x = legendre_points(n)
        else:
            x = fourier_points(n, (domains[d] if domains else (0.0, 2 * np.pi)))
        shp = [1] * nd
        shp[d] = n
        out.append(x.reshape(shp))
    return out


# ---- manufactured solutions -----------------------------------------------------------
def poisson2d_u(x, y):
    return np.sin(np.pi * x) * (1 + np.cos(2 * y) + np.sin(3 * y))


def poisson2d_f(x, y):
    """-lap(u) for poisson2d_u."""
    p2 = np.pi ** 2
    return np.sin(np.pi * x) * (p2 + (p2 + 4) * np.cos(2 * y) + (p2 + 9) * np.sin(3 * y))


def box3d_u(x, y, z):
    return (1 - x ** 2) ** 2 * np.sin(y) * np.cos(2 * z)


def box3d_f_poisson(x, y, z):
    """-lap(u) for box3d_u."""
    return (9 - 22 * x ** 2 + 5 * x ** 4) * np.sin(y) * np.cos(2 * z)


def box3d_f_biharmonic(x, y, z):
    """lap^2(u) for box3d_u."""
    return (89 - 170 * x ** 2 + 25 * x ** 4) * np.sin(y) * np.cos(2 * z)


# ---- random data ----------------------------------------------------------------------------
def signed_index(M, r2c=False):
    if r2c:
        return np.arange(M // 2 + 1, dtype=np.float64)
    l = np.arange(M, dtype=np.float64)
    return np.where(l < (M + 1) // 2, l, l - M)


def coefficients(kinds, sizes, scale, workload="box3d", item=0, nvalid0=None, dtype=np.complex128):
    """Complex N(0,1) * exp(-|k|/scale) on the stored spectral shape.

    Rows nvalid0.. of axis 0 (past the Shen basis size) are zero.
    """
    g = rng(workload, item)
    shp = list(sizes)
    if kinds[-1] == "r2c":
        shp[-1] = sizes[-1] // 2 + 1
    knorm2 = np.zeros(shp)
    for d, (k, n) in enumerate(zip(kinds, sizes)):
        if k in ("chebyshev", "dirichlet", "neumann", "biharmonic"):
            idx = np.arange(n, dtype=np.float64)
        else:
            idx = signed_index(n, k == "r2c")
        v = [1] * len(shp)
        v[d] = -1
        knorm2 = knorm2 + (idx ** 2).reshape(v)
    c = (g.standard_normal(shp) + 1j * g.standard_normal(shp)) * np.exp(-np.sqrt(knorm2) / scale)
    if nvalid0 is not None:
        c[nvalid0:] = 0
    return c.astype(dtype)


def gl_initial(M, item=0):
    g = rng("gl", item)
    return 0.01 * (g.standard_normal((M, M)) + 1j * g.standard_normal((M, M)))


def batch1d(nprob=4096, item=0, nmin=16, nmax=2048):
    """Sizes, alphas and physical right-hand sides of the batched 1D Helmholtz problems."""
    g = rng("batch", item)
    sizes = np.rint(np.exp(g.uniform(np.log(nmin), np.log(nmax), nprob))).astype(np.int64)
    alpha = g.uniform(0.0, 1e4, nprob)
    fs = []
    for N in sizes:
        c = g.standard_normal(N) * np.exp(-8.0 * np.arange(N) / N)
        fs.append(npcheb.chebval(cheb_points(N), c))
    return sizes, alpha, fs


BATCH2D_SIDES = (64, 128, 256, 512, 1024)


def batch2d(nprob=64, item=0, sides=BATCH2D_SIDES, modes=16):
    """Sizes and physical right-hand sides of the batched 2-D problems: square N x N grids
    (Shen-Dirichlet x R2C Fourier on [-1, 1] x [0, 2 pi)), N uniform over `sides`;
    f = Re sum_{k, l < modes} c_kl T_k(x) exp(i l y), c_kl ~ N(0,1) + i N(0,1) times
    exp(-(k + l) / 4)."""
    g = rng("batch", 500 + item)
    sizes = [(int(N), int(N)) for N in g.choice(np.asarray(sides), nprob)]
    fs = []
    k = np.arange(modes)
    for N, M in sizes:
        c = (g.standard_normal((modes, modes)) + 1j * g.standard_normal((modes, modes))) * np.exp(
            -(k[:, None] + k[None, :]) / 4.0)
        Tx = np.cos(np.outer(np.arccos(cheb_points(N)), k))     # T_k(x_j)
        Ey = np.exp(1j * np.outer(k, fourier_points(M)))         # exp(i l y_m)
        fs.append(np.real(Tx @ c @ Ey))
    return sizes, fs

