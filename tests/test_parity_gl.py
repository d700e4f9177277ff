"""GPU parity of the Ginzburg-Landau stepper (Sec. 6) against the FP64 oracle.

Tolerances (relative L2 over the spectral array): f64 1e-12 for the right-hand side and one
step, 1e-11 after 10 steps; f32 (complex64 state, FP32 arithmetic) 2e-5 for the right-hand
side and one step.
"""
import numpy as np
import pytest
import torch

from oracle import fourier
from oracle import ginzburg_landau as ogl
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
DOMAIN = [(-50.0, 50.0), (-50.0, 50.0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def make(M, prec, beta, gamma, dt, scheme):
    from paper_1708_03188_gb300.sgm import GinzburgLandau, Space
    sp = Space(["c2c", "c2c"], (M, M), domain=DOMAIN, precision=prec)
    return sp, GinzburgLandau(sp, beta, gamma, dt, scheme)


def smooth_state(M, item=0, amp=0.02):
    """Decaying random spectrum whose physical field is O(1) (sum of |coefficients| ~ 1)."""
    g = inputs.rng("gl", 50 + item)
    l = fourier.wavenumbers(M)
    k = np.sqrt(l[:, None] ** 2 + l[None, :] ** 2)
    return amp * (g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))) * np.exp(-k / 4.0)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(x, gl):
    return torch.from_numpy(np.ascontiguousarray(x)).to(gl.dtype).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("M", [32, 64])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("beta,gamma", [(1.5, -0.5), (0.0, 1.5)])
def test_rhs(M, prec, tol, beta, gamma):
    _, gl = make(M, prec, beta, gamma, 0.01, "rk4")
    u = dev(smooth_state(M), gl)
    ref = ogl.rhs(host(u), beta, gamma)
    assert rel(host(gl.rhs(u)), ref) < tol


@pytest.mark.parametrize("scheme,ostep", [("rk4", ogl.rk4_step), ("ifrk4", ogl.if_rk4_step)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_one_step(scheme, ostep, prec, tol):
    M, beta, gamma, dt = 64, 1.5, -0.5, 0.01
    _, gl = make(M, prec, beta, gamma, dt, scheme)
    u = dev(smooth_state(M, 1), gl)
    ref = ostep(host(u), dt, beta, gamma)
    assert rel(host(gl.step(u, 1)), ref) < tol


@pytest.mark.parametrize("scheme,ostep", [("rk4", ogl.rk4_step), ("ifrk4", ogl.if_rk4_step)])
def test_ten_steps_f64(scheme, ostep):
    M, beta, gamma, dt = 32, 1.5, -0.5, 0.05
    _, gl = make(M, "f64", beta, gamma, dt, scheme)
    u = dev(smooth_state(M, 2), gl)
    ref = host(u)
    for _ in range(10):
        ref = ostep(ref, dt, beta, gamma)
    assert rel(host(gl.step(u, 10)), ref) < 1e-11


def test_plane_wave_exact():
    # u = A exp(i(k.x - w t)), |A|^2 = 1 - |k|^2, w = beta |k|^2 + gamma (1 - |k|^2)
    M, beta, gamma, T, n = 64, 1.5, -0.5, 1.0, 40
    k0, k1 = 2 * np.pi * 3 / 100, 2 * np.pi * 2 / 100
    k2 = k0 * k0 + k1 * k1
    A, om = np.sqrt(1 - k2), beta * k2 + gamma * (1 - k2)
    x = -50 + 100 * np.arange(M) / M
    wave = lambda t: A * np.exp(1j * (k0 * (x[:, None] + 50) + k1 * (x[None, :] + 50) - om * t))
    to_hat = lambda u: fourier.c2c_forward(fourier.c2c_forward(u, 0), 1)
    for scheme in ("rk4", "ifrk4"):
        _, gl = make(M, "f64", beta, gamma, T / n, scheme)
        u = dev(to_hat(wave(0.0)), gl)
        assert rel(host(gl.step(u, n)), to_hat(wave(T))) < 1e-6


def test_real_initial_condition_keeps_symmetry():
    # Sec. 6: (x + y) exp(-0.03 (x^2 + y^2)) keeps u(x, y) = u(y, x) with de-aliasing.
    M = 64
    x = -50 + 100 * np.arange(M) / M
    u0 = (x[:, None] + x[None, :]) * np.exp(-0.03 * (x[:, None] ** 2 + x[None, :] ** 2))
    _, gl = make(M, "f64", 0.0, 1.5, 0.025, "rk4")
    u = dev(fourier.c2c_forward(fourier.c2c_forward(u0.astype(complex), 0), 1), gl)
    uh = host(gl.step(u, 40))
    assert np.max(np.abs(uh - uh.T)) < 1e-12 * np.max(np.abs(uh))


def test_argument_errors():
    from paper_1708_03188_gb300.sgm import GinzburgLandau, SgmError, Space
    sp = Space(["c2c", "c2c"], (48, 48), domain=DOMAIN, precision="f64")
    with pytest.raises(SgmError):
        GinzburgLandau(sp, 1.5, -0.5, 0.01)                 # size without kernels
    sp = Space(["c2c", "c2c"], (64, 64), domain=DOMAIN, precision="f64")
    with pytest.raises(SgmError):
        GinzburgLandau(sp, 1.5, -0.5, 0.01, padding=2.0)
    with pytest.raises(SgmError):
        GinzburgLandau(sp, 1.5, -0.5, -0.01)
    sp3 = Space(["dirichlet", "c2c"], (16, 64), precision="f64")
    with pytest.raises(SgmError):
        GinzburgLandau(sp3, 1.5, -0.5, 0.01)
