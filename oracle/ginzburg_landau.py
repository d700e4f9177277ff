"""Complex Ginzburg-Landau right-hand side and RK4 steppers (oracle).

Sec. 6 of the paper solves u_t = lap(u) + u - (1 + 1.5i) u |u|^2 on the doubly
periodic [-50, 50]^2 with Fourier bases mapped onto [0, 2 pi).  The equation is
taken here in the general form
    u_t = u + (1 + i beta) lap(u) - (1 + i gamma) |u|^2 u
(the paper's form is beta = 0, gamma = 1.5).  In Fourier space (Eq. Ginz_var,
after dividing by the Fourier mass factor (2 pi)^2):
    du_hat/dt = L(k) u_hat - N(u_hat),   L(k) = 1 - (1 + i beta) |k|^2,
with |k|^2 built from k = 2 pi l / 100 on each axis.  The nonlinear term uses
the padded transforms of Sec. 6: the coefficients are copied into a larger
spectral array (padding factor 3/2, wavenumber l keeps its value, the rest is
zero), transformed back without scaling, multiplied pointwise, transformed
forward with 1/Mp per axis and truncated to the original wavenumber set.

Steppers:
  rk4_step     the paper's explicit classical RK4 (Sec. 6, the RK coefficients
               a = [1/6, 1/3, 1/3, 1/6], b = [1/2, 1/2, 1]).
  if_rk4_step  integrating-factor RK4: the same classical RK4 applied to
               v = exp(-L t) u_hat, so the linear diagonal term is integrated
               exactly (Lawson's form).  Used where the explicit scheme's
               stability limit is below the requested time step.
All dense: every transform is an explicit DFT matrix product.
"""
import numpy as np

from . import fourier


def padded_size(M, factor):
    return int(np.floor(factor * M + 1e-9))


def pad(u_hat, Mp):
    """Copy wavenumber l of each axis to the same wavenumber of the padded array."""
    M0, M1 = u_hat.shape
    out = np.zeros((Mp, Mp), dtype=np.complex128)
    l0 = fourier.wavenumbers(M0).astype(int) % Mp
    l1 = fourier.wavenumbers(M1).astype(int) % Mp
    out[np.ix_(l0, l1)] = u_hat
    return out


def truncate(up_hat, M):
    Mp = up_hat.shape[0]
    l = fourier.wavenumbers(M).astype(int) % Mp
    return up_hat[np.ix_(l, l)]


def padded_backward(u_hat, Mp):
    """Physical values on the padded Mp x Mp mesh (backward sums, no scaling)."""
    return fourier.c2c_backward(fourier.c2c_backward(pad(u_hat, Mp), 0), 1)


def padded_forward_truncated(g, M):
    """Forward transform on the padded mesh (1/Mp per axis), truncated to M x M."""
    return truncate(fourier.c2c_forward(fourier.c2c_forward(g, 0), 1), M)


def nonlinear(u_hat, gamma, padding=1.5):
    """N(u_hat) = truncated forward transform of (1 + i gamma) |u|^2 u on the padded mesh."""
    M = u_hat.shape[0]
    Mp = padded_size(M, padding)
    up = padded_backward(u_hat, Mp)
    return padded_forward_truncated((1.0 + 1j * gamma) * up * np.abs(up) ** 2, M)


def linear_symbol(M, beta, L=100.0):
    """L(k) = 1 - (1 + i beta) |k|^2 with k = 2 pi l / L on each axis."""
    k = fourier.wavenumbers(M) * (2 * np.pi / L)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    return 1.0 - (1.0 + 1j * beta) * k2


def rhs(u_hat, beta, gamma, padding=1.5, L=100.0):
    """du_hat/dt = L(k) u_hat - N(u_hat)."""
    return linear_symbol(u_hat.shape[0], beta, L) * u_hat - nonlinear(u_hat, gamma, padding)


def rk4_step(u_hat, dt, beta, gamma, padding=1.5, L=100.0):
    """One explicit classical RK4 step in the order of the paper's time loop (Sec. 6)."""
    a = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
    b = (0.5, 0.5, 1.0)
    u0 = u_hat.copy()
    u1 = u_hat.copy()
    u = u_hat.copy()
    for rk in range(4):
        du = rhs(u, beta, gamma, padding, L)
        if rk < 3:
            u = u0 + b[rk] * dt * du
        u1 = u1 + a[rk] * dt * du
    return u1


def if_rk4_step(u_hat, dt, beta, gamma, padding=1.5, L=100.0):
    """Classical RK4 on v = exp(-L t) u_hat (integrating factor, Lawson form)."""
    Lk = linear_symbol(u_hat.shape[0], beta, L)
    E = np.exp(0.5 * dt * Lk)
    N = lambda v: -nonlinear(v, gamma, padding)
    k1 = N(u_hat)
    k2 = N(E * (u_hat + 0.5 * dt * k1))
    k3 = N(E * u_hat + 0.5 * dt * k2)
    k4 = N(E * E * u_hat + dt * E * k3)
    return E * E * u_hat + dt / 6.0 * (E * E * k1 + 2.0 * E * (k2 + k3) + k4)
