"""GPU parity of the streaming pipeline (TMA-fed persistent transform kernels, padded FP32/FP64
intermediates; used by the physical-to-physical solves of FP32 spaces with a Shen axis of 64,
128 or 256 points, a strided C2C axis of 32..256 and an even R2C axis of 64..1024) against the FP64
oracle: the full chain scalar product -> dense LU per column -> backward sum on a random
right-hand side, for each Shen basis, 2-D and 3-D, square and non-square Fourier boxes (the
four-column biharmonic grouping needs the square one).  Tolerance 2e-5 relative L2 (FP32
transforms, FP64 eliminations, as the manufactured FP32 solves).
"""
import numpy as np
import pytest
import torch

from oracle.space import Space as OSpace
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [(["dirichlet", "r2c"], [64, 64], (-1.0, 0.0)),
         (["biharmonic", "r2c"], [128, 128], (1.0, 0.0, 0.0)),
         (["dirichlet", "c2c", "r2c"], [64, 32, 64], (-1.0, 0.0)),
         (["dirichlet", "c2c", "r2c"], [128, 64, 64], (1.0, -100.0)),
         (["biharmonic", "c2c", "r2c"], [64, 32, 32 * 2], (1.0, 0.0, 0.0)),
         (["biharmonic", "c2c", "r2c"], [64, 64, 64], (1.0, -2.0, 5.0)),
         (["neumann", "c2c", "r2c"], [128, 32, 64], (1.0, -30.0))]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


@pytest.mark.parametrize("kinds,sizes,coef", CASES)
def test_stream_solve_against_oracle(kinds, sizes, coef):
    from paper_1708_03188_gb300.sgm import Space, tc_wait_timeouts
    sp = Space(kinds, sizes, precision="f32")
    osp = OSpace(kinds, sizes)
    g = inputs.rng("box3d", 870 + len(kinds) + sizes[0])
    f = torch.from_numpy(g.standard_normal(sizes)).float().cuda()
    fo = f.cpu().double().numpy()
    if kinds[0] == "biharmonic":
        got = sp.biharmonic(*coef, f)
        ref = osp.backward(osp.biharmonic(*coef, osp.scalar_product(fo)))
    else:
        got = sp.helmholtz(*coef, f)
        ref = osp.backward(osp.helmholtz(*coef, osp.scalar_product(fo)))
    got = got.cpu().double().numpy()
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"stream {kinds} {sizes}: {e:.2e}")
    assert e < 2e-5
    assert tc_wait_timeouts() == 0
    sp.close()


@pytest.mark.parametrize("kinds,sizes", [(["biharmonic", "c2c", "r2c"], [64, 64, 64]),
                                         (["dirichlet", "c2c", "r2c"], [64, 32, 64])])
def test_solve_events_bracket_the_elimination(kinds, sizes):
    """sgm_space_solve_events: the events are recorded around the elimination of every solve
    until cleared, the elimination takes a positive part of the solve, and the result is the
    one without events."""
    from paper_1708_03188_gb300.sgm import SgmError, Space
    sp = Space(kinds, sizes, precision="f32")
    g = inputs.rng("box3d", 880 + sizes[0])
    f = torch.from_numpy(g.standard_normal(sizes)).float().cuda()
    solve = (lambda: sp.biharmonic(1.0, 0.0, 0.0, f)) if kinds[0] == "biharmonic" else \
        (lambda: sp.helmholtz(-1.0, 0.0, f))
    plain = solve()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sp.solve_events(a, b)
    t0.record()
    got = solve()
    t1.record()
    torch.cuda.synchronize()
    inner, outer = a.elapsed_time(b), t0.elapsed_time(t1)
    assert 0.0 < inner <= outer
    assert torch.equal(got, plain)
    sp.solve_events()
    with pytest.raises(SgmError):
        sp.solve_events(a, None)
    sp.close()
