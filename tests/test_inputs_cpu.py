"""CPU checks of the seeded input recipes (paper_1708_03188_gb300/inputs.py).

The manufactured right-hand sides are checked against central finite differences of their exact
solutions at random points, independently of the closed forms. The seeded generators are
checked for determinism and for the shapes and ranges of their recipes.
"""
import numpy as np
import pytest

from paper_1708_03188_gb300 import inputs


def lap2(fun, x, y, h=1e-3):
    return (fun(x + h, y) + fun(x - h, y) + fun(x, y + h) + fun(x, y - h) - 4 * fun(x, y)) / h ** 2


def lap3(fun, x, y, z, h=1e-3):
    c = fun(x, y, z)
    return (fun(x + h, y, z) + fun(x - h, y, z) + fun(x, y + h, z) + fun(x, y - h, z) + fun(x, y, z + h)
            + fun(x, y, z - h) - 6 * c) / h ** 2


def test_poisson2d_pair_is_minus_laplacian():
    g = np.random.default_rng(1)
    x, y = g.uniform(-0.9, 0.9, 50), g.uniform(0, 2 * np.pi, 50)
    fd = -lap2(inputs.poisson2d_u, x, y)
    assert np.max(np.abs(fd - inputs.poisson2d_f(x, y))) < 1e-4 * np.max(np.abs(fd))


def test_box3d_pairs_are_minus_laplacian_and_bilaplacian():
    g = np.random.default_rng(2)
    x, y, z = g.uniform(-0.9, 0.9, 40), g.uniform(0, 2 * np.pi, 40), g.uniform(0, 2 * np.pi, 40)
    fp = -lap3(inputs.box3d_u, x, y, z)
    assert np.max(np.abs(fp - inputs.box3d_f_poisson(x, y, z))) < 1e-4 * np.max(np.abs(fp))
    # lap^2 u = lap(lap u), with lap u = -f_poisson in closed form: one finite-difference level
    fb = lap3(lambda a, b, c: -inputs.box3d_f_poisson(a, b, c), x, y, z)
    assert np.max(np.abs(fb - inputs.box3d_f_biharmonic(x, y, z))) < 1e-4 * np.max(np.abs(fb))


def test_box3d_solution_vanishes_with_its_normal_derivative():
    y, z = np.linspace(0, 6, 7), np.linspace(0, 6, 7)
    for xb in (-1.0, 1.0):
        assert np.max(np.abs(inputs.box3d_u(xb, y, z))) == 0.0
        h = 1e-6
        du = (inputs.box3d_u(xb + h, y, z) - inputs.box3d_u(xb - h, y, z)) / (2 * h)
        assert np.max(np.abs(du)) < 1e-9


def test_seeded_generators_are_deterministic():
    s1, a1, f1 = inputs.batch1d(64)
    s2, a2, f2 = inputs.batch1d(64)
    assert np.array_equal(s1, s2) and np.array_equal(a1, a2)
    assert all(np.array_equal(p, q) for p, q in zip(f1, f2))
    t1, g1 = inputs.batch2d(8)
    t2, g2 = inputs.batch2d(8)
    assert t1 == t2 and all(np.array_equal(p, q) for p, q in zip(g1, g2))
    assert np.array_equal(inputs.gl_initial(32, 3), inputs.gl_initial(32, 3))
    assert not np.array_equal(inputs.gl_initial(32, 3), inputs.gl_initial(32, 4))


def test_batch_recipes():
    sizes, alpha, fs = inputs.batch1d(4096)
    assert sizes.min() >= 16 and sizes.max() <= 2048
    assert alpha.min() >= 0 and alpha.max() <= 1e4
    assert [len(f) for f in fs] == list(sizes)
    # log-uniform: about half of the sizes below the geometric midpoint sqrt(16 * 2048) = 181
    assert 0.45 < np.mean(sizes < 181) < 0.55
    sizes2d, fs2 = inputs.batch2d(64)
    assert len(sizes2d) == 64 and all(N == M and N in inputs.BATCH2D_SIDES for N, M in sizes2d)
    assert all(f.shape == s for f, s in zip(fs2, sizes2d)) and all(np.isfinite(f).all() for f in fs2)


@pytest.mark.parametrize("M", [32, 64])
def test_gl_initial_amplitude(M):
    u = inputs.gl_initial(M, 0)
    assert u.shape == (M, M) and np.iscomplexobj(u)
    # 0.01 (N(0,1) + i N(0,1)): mean square 2e-4
    assert 1e-4 < np.mean(np.abs(u) ** 2) < 3e-4
