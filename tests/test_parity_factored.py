"""GPU parity of the factored eliminations of 3-D spaces against the FP64 oracle.

A 3-D Shen-Dirichlet or Shen-biharmonic space stores the FP64 factorisation of each operator
(a, b, c) it solves in one of two slots and replays it for later solves with the same
coefficients (least recently used slot replaced).  Checked here, each result against the
oracle's dense LU per column:
  - repeated coefficients (slot hits), three alternating operators (replacement) and the mass
    solve of the forward transform in between, on square and non-square Fourier boxes with even
    and odd lengths along axis 1 (the table entry of a pair of columns +-l1 serves both; the
    columns l1 = 0 and, for even lengths, l1 = -M1/2 have their own), FP64 and FP32;
  - the spectral column layout (sgm_helmholtz_solve) and the padded layout of the streaming
    physical-to-physical solve (sgm_helmholtz) alternating on one FP32 space;
  - a solve captured in a CUDA graph (inside a capture the self-contained elimination kernels
    run) replayed after eager solves that replaced both slots.
Tolerances: FP64 max(1e-12, 32 * 2^-53 * cond) relative L2, cond the largest condition number of
the column systems; FP32 spectral 2e-6; FP32 physical to physical 2e-5.
"""
import numpy as np
import pytest
import torch

from oracle import galerkin
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


def gspace(kinds, sizes, prec):
    from paper_1708_03188_gb300.sgm import Space
    return Space(kinds, sizes, precision=prec)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rhs(gs, nb, item):
    g = inputs.rng("box3d", 940 + item)
    f = g.standard_normal(gs.spectral_shape) + 1j * g.standard_normal(gs.spectral_shape)
    f[nb:] = 0
    fd = torch.from_numpy(f).to(gs.spectral_dtype).cuda()
    return fd, to_np(fd)


def tolerance(os_, kind, coef, prec):
    if prec == "f32":
        return 2e-6
    mats = os_.matrices()
    k2 = np.atleast_1d(os_.kappa2()).ravel()
    if kind == "dirichlet":
        cond = max(np.linalg.cond(galerkin.helmholtz_matrix(mats, *coef, v)) for v in k2)
    else:
        cond = max(np.linalg.cond(galerkin.biharmonic_matrix(mats, *coef, v)) for v in k2)
    return max(1e-12, 32 * EPS * cond)


def solve(gs, os_, kind, coef, fd, fo):
    if kind == "dirichlet":
        return to_np(gs.helmholtz_solve(*coef, fd)), os_.helmholtz(*coef, fo)
    return to_np(gs.biharmonic_solve(*coef, fd)), os_.biharmonic(*coef, fo)


OPS = {"dirichlet": [(-1.0, 0.0), (1.0, -300.0), (0.5, 2.0)],
       "biharmonic": [(1.0, 0.0, 0.0), (1.3, -0.4, 2.0), (0.0, 1.0, -5.0)]}
# operator index per call: hits, a third operator replacing the least recently used slot, and
# the return of an evicted one
SEQUENCE = [0, 0, 1, 0, 2, 1, 0, 2, 2]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("kinds,sizes", [(["dirichlet", "c2c", "r2c"], [24, 40, 64]),
                                         (["dirichlet", "c2c", "r2c"], [24, 16, 16]),
                                         (["biharmonic", "c2c", "r2c"], [32, 16, 16]),
                                         (["biharmonic", "c2c", "r2c"], [32, 33, 34]),
                                         (["dirichlet", "c2c", "r2c"], [20, 9, 12])],
                         ids=lambda v: "-".join(map(str, v)))
def test_slot_hits_and_replacement(kinds, sizes, prec):
    kind = kinds[0]
    nb = sizes[0] - (2 if kind == "dirichlet" else 4)
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    tols = [tolerance(os_, kind, c, prec) for c in OPS[kind]]
    x = inputs.rng("box3d", 939).standard_normal(gs.physical_shape)
    xd = torch.from_numpy(x).to(gs.physical_dtype).cuda()
    xo = xd.cpu().double().numpy()
    condB = np.linalg.cond(os_.matrices()["B"])
    ftol = (1e-12 if prec == "f64" else 4e-6) * max(1.0, condB)
    for step, op in enumerate(SEQUENCE):
        fd, fo = rhs(gs, nb, step)
        got, ref = solve(gs, os_, kind, OPS[kind][op], fd, fo)
        assert np.all(got[nb:] == 0)
        assert rel(got, ref) < tols[op], (step, op, rel(got, ref))
        if step in (1, 4):
            # the forward transform's mass solve is a fourth operator in the same slots
            assert rel(to_np(gs.forward(xd)), os_.forward(xo)) < ftol
    gs.close()


@pytest.mark.parametrize("kinds,sizes,coef", [(["dirichlet", "c2c", "r2c"], [64, 32, 64], (-1.0, 0.0)),
                                              (["biharmonic", "c2c", "r2c"], [64, 32, 32], (1.0, 0.0, 0.0))])
def test_spectral_and_streaming_layouts_alternate(kinds, sizes, coef):
    """The padded streaming intermediates and the spectral arrays give two column layouts of the
    same operator; each has its own slot key."""
    kind = kinds[0]
    nb = sizes[0] - (2 if kind == "dirichlet" else 4)
    gs = gspace(kinds, sizes, "f32")
    os_ = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 960)
    for rep in range(3):
        f = torch.from_numpy(g.standard_normal(sizes)).float().cuda()
        fo = f.cpu().double().numpy()
        if kind == "dirichlet":
            got = gs.helmholtz(*coef, f).cpu().double().numpy()
            ref = os_.backward(os_.helmholtz(*coef, os_.scalar_product(fo)))
        else:
            got = gs.biharmonic(*coef, f).cpu().double().numpy()
            ref = os_.backward(os_.biharmonic(*coef, os_.scalar_product(fo)))
        assert rel(got, ref) < 2e-5, (rep, rel(got, ref))
        fd, fho = rhs(gs, nb, 970 + rep)
        got, ref = solve(gs, os_, kind, coef, fd, fho)
        assert rel(got, ref) < 2e-6, (rep, rel(got, ref))
    gs.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_captured_solve_after_slots_replaced(prec):
    kinds, sizes = ["dirichlet", "c2c", "r2c"], [24, 16, 32]
    gs = gspace(kinds, sizes, prec)
    os_ = OSpace(kinds, sizes)
    fd, fo = rhs(gs, 22, 980)
    out = torch.empty_like(fd)
    a1, a2, a3 = OPS["dirichlet"]
    gs.helmholtz_solve(*a1, fd, out=out)   # eager: a1 in a slot
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gs.helmholtz_solve(*a1, fd, out=out)
    # eager solves with two other operators evict a1 from both slots
    for c in (a2, a3):
        got, ref = solve(gs, os_, "dirichlet", c, *rhs(gs, 22, 981))
        assert rel(got, ref) < tolerance(os_, "dirichlet", c, prec)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    ref = os_.helmholtz(*a1, fo)
    assert rel(to_np(out), ref) < tolerance(os_, "dirichlet", a1, prec)
    # and an eager a1 afterwards refactors into a slot
    got, ref = solve(gs, os_, "dirichlet", a1, fd, fo)
    assert rel(got, ref) < tolerance(os_, "dirichlet", a1, prec)
    del graph
    gs.close()
