"""Dense discrete Fourier transforms (oracle, test infrastructure).

Sec. 3.4.1 of the paper: on the mesh X_j = 2 pi j / M the forward transform is
  u_hat_l = (1/M) sum_j u_j exp(-i l X_j)
and the backward transform (no 1/M) is
  u_j = sum_l u_hat_l exp(i l X_j).
A physical domain [a, a+L) is mapped onto [0, 2 pi) (Sec. 6), so wavenumbers
enter derivatives as k = 2 pi l / L.  Coefficients are kept in the usual FFT
order l = 0, 1, ..., -2, -1; a real-to-complex axis keeps l = 0..floor(M/2)
(Sec. 3.4.1, the symmetry u_hat_k = conj(u_hat_{M-k}) of real data).
Every transform here is an explicit O(M^2) matrix product, not an FFT.
"""
import numpy as np


def wavenumbers(M, r2c=False):
    """Integer wavenumbers of the stored coefficients, FFT order."""
    if r2c:
        return np.arange(M // 2 + 1, dtype=np.float64)
    l = np.arange(M, dtype=np.float64)
    return np.where(l < (M + 1) // 2, l, l - M)    # even M: index M/2 -> -M/2


def dft_matrix(M, sign):
    """E[l, j] = exp(sign * i * l * X_j) for the C2C wavenumber set."""
    l = wavenumbers(M)
    X = 2.0 * np.pi * np.arange(M) / M
    return np.exp(sign * 1j * np.outer(l, X))


def _apply(mat, u, axis):
    u = np.moveaxis(np.asarray(u), axis, 0)
    out = np.tensordot(mat, u, axes=([1], [0]))
    return np.moveaxis(out, 0, axis)


def c2c_forward(u, axis):
    """u_hat_l = (1/M) sum_j u_j exp(-i l X_j) along ``axis``."""
    M = np.shape(u)[axis]
    return _apply(dft_matrix(M, -1.0) / M, u, axis)


def c2c_backward(u_hat, axis):
    """u_j = sum_l u_hat_l exp(i l X_j) along ``axis`` (no scaling)."""
    M = np.shape(u_hat)[axis]
    return _apply(dft_matrix(M, +1.0).T, u_hat, axis)


def r2c_forward(u, axis):
    """Real input: keep l = 0..floor(M/2) of the C2C forward transform."""
    M = np.shape(u)[axis]
    full = c2c_forward(np.asarray(u, dtype=np.complex128), axis)
    return np.take(full, np.arange(M // 2 + 1), axis=axis)


def hermitian_extend(u_hat, M, axis):
    """Full C2C coefficient set from the l = 0..floor(M/2) half of real data."""
    u_hat = np.moveaxis(np.asarray(u_hat, dtype=np.complex128), axis, 0)
    full = np.zeros((M,) + u_hat.shape[1:], dtype=np.complex128)
    h = M // 2 + 1
    full[:h] = u_hat
    for n in range(h, M):
        full[n] = np.conj(u_hat[M - n])
    return np.moveaxis(full, 0, axis)


def c2r_backward(u_hat, M, axis):
    """Real part of the backward sum over the Hermitian-extended coefficients.

    The imaginary parts of the self-conjugate entries (l = 0, and l = M/2 for
    even M) do not reach the real result, as for any real-data inverse DFT.
    """
    return c2c_backward(hermitian_extend(u_hat, M, axis), axis).real
