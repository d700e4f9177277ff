"""GPU checks of the Ginzburg-Landau stepper at the timed size: 512^2 on [-50, 50]^2, padded to
768^2, beta = 1.5, gamma = -0.5, with the two schemes and step sizes the benchmark times
(integrating-factor RK4 at dt = 0.01, explicit RK4 at dt = 0.0025).  The dense-DFT oracle is too
slow at this size, so the checks use properties that hold at any size:
  - the plane wave u = A exp(i(k.x - w t)), |A|^2 = 1 - |k|^2, w = beta |k|^2 + gamma (1 - |k|^2),
    an exact solution (a single mode does not alias), FP64 to T = 1: tolerance 1e-6 as at 64^2,
    where the steps were larger;
  - complex64 against complex128 after one step from the benchmark's seeded state: tolerance
    2e-5, the FP32 one-step tolerance against the oracle at 32^2 and 64^2.
"""
import numpy as np
import pytest
import torch

from oracle import fourier
from paper_1708_03188_gb300 import inputs

pytestmark = pytest.mark.gpu
M = 512
DOMAIN = [(-50.0, 50.0), (-50.0, 50.0)]
SCHEMES = [("ifrk4", 0.01), ("rk4", 0.0025)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1708_03188_gb300 import build
    build.build()


def make(prec, dt, scheme):
    from paper_1708_03188_gb300.sgm import GinzburgLandau, Space
    sp = Space(["c2c", "c2c"], (M, M), domain=DOMAIN, precision=prec)
    return sp, GinzburgLandau(sp, 1.5, -0.5, dt, scheme)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("scheme,dt", SCHEMES)
def test_plane_wave_512(scheme, dt):
    beta, gamma, T = 1.5, -0.5, 1.0
    k0, k1 = 2 * np.pi * 3 / 100, 2 * np.pi * 2 / 100
    k2 = k0 * k0 + k1 * k1
    A, om = np.sqrt(1 - k2), beta * k2 + gamma * (1 - k2)
    x = -50 + 100 * np.arange(M) / M
    wave = lambda t: A * np.exp(1j * (k0 * (x[:, None] + 50) + k1 * (x[None, :] + 50) - om * t))
    to_hat = lambda u: np.ascontiguousarray(fourier.c2c_forward(fourier.c2c_forward(u, 0), 1))
    sp, gl = make("f64", dt, scheme)
    u = torch.from_numpy(to_hat(wave(0.0))).cuda()
    n = int(round(T / dt))
    out = gl.step(u, n).cpu().numpy()
    e = rel(out, to_hat(wave(n * dt)))
    print(f"plane wave 512^2 {scheme} dt={dt}: {e:.2e}")
    assert e < 1e-6
    gl.close()
    sp.close()


@pytest.mark.parametrize("scheme,dt", SCHEMES)
def test_complex64_against_complex128_one_step_512(scheme, dt):
    u0 = inputs.gl_initial(M)
    out = {}
    for prec in ("f64", "f32"):
        sp, gl = make(prec, dt, scheme)
        u = sp.forward(torch.from_numpy(u0).to(sp.physical_dtype).cuda())
        out[prec] = gl.step(u, 1).cpu().numpy().astype(np.complex128)
        gl.close()
        sp.close()
    e = rel(out["f32"], out["f64"])
    print(f"complex64 vs complex128, one {scheme} step at 512^2: {e:.2e}")
    assert e < 2e-5
