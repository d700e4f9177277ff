"""Tensor-product spaces: scalar product, forward, backward, solves (oracle).

Sec. 4 of the paper: a space is one Chebyshev (Shen) axis, axis 0, times any
number of Fourier axes, or Fourier axes only.  Transform order (Sec. 4, the
right-hand-side formula after Eq. laplace): the forward direction applies the
Fourier transforms first (real-to-complex on the last axis, then the
complex-to-complex axes from last to first) and the Shen scalar product
  S_l(u) = (u, phi_l)_w^N = sum_j u(x_j) phi_l(x_j) w_j        (Sec. 3.4.2)
last; the backward direction is the reverse, with the Shen backward sum
  u(x_j) = sum_l u_hat_l phi_l(x_j)                            (Eq. fast_shen).
The forward transform is the projection u_hat = B^{-1} S(u)  (Sec. 3.4.2).

Stored spectral layout: axis 0 keeps all N rows, the rows past the basis size
(2 for Dirichlet, 4 for biharmonic) are zero; Fourier axes are in FFT order,
the last one halved when real-to-complex.
"""
import numpy as np

from . import fourier, galerkin, quadrature

FOURIER = ("c2c", "r2c")


class Space:
    def __init__(self, kinds, sizes, domains=None):
        self.kinds = tuple(kinds)
        self.sizes = tuple(int(n) for n in sizes)
        assert len(self.kinds) == len(self.sizes)
        self.has_cheb = self.kinds[0] in quadrature.KINDS
        for d, k in enumerate(self.kinds):
            if d == 0 and self.has_cheb:
                continue
            assert k in FOURIER, k
            assert k == "c2c" or d == len(self.kinds) - 1, "only the last axis may be r2c"
        if domains is None:
            domains = [(-1.0, 1.0) if (d == 0 and self.has_cheb) else (0.0, 2 * np.pi)
                       for d in range(len(self.kinds))]
        self.domains = [tuple(map(float, dm)) for dm in domains]
        self.real = self.kinds[-1] == "r2c" or (self.has_cheb and len(self.kinds) == 1)
        self._mats = None

    # ---- shapes -----------------------------------------------------------------
    @property
    def physical_shape(self):
        return self.sizes

    @property
    def spectral_shape(self):
        s = list(self.sizes)
        if self.kinds[-1] == "r2c":
            s[-1] = s[-1] // 2 + 1
        return tuple(s)

    @property
    def fourier_axes(self):
        return [d for d in range(len(self.kinds)) if self.kinds[d] in FOURIER]

    def kappa2(self):
        """Sum over Fourier axes of (2 pi l / L)^2, shaped like one axis-0 slice."""
        shp = self.spectral_shape
        start = 1 if self.has_cheb else 0
        k2 = np.zeros(shp[start:])
        for d in range(start, len(shp)):
            M = self.sizes[d]
            L = self.domains[d][1] - self.domains[d][0]
            k = fourier.wavenumbers(M, r2c=self.kinds[d] == "r2c") * (2 * np.pi / L)
            view = [1] * (len(shp) - start)
            view[d - start] = -1
            k2 = k2 + (k ** 2).reshape(view)
        return k2

    def matrices(self):
        if self._mats is None:
            self._mats = galerkin.matrices(self.kinds[0], self.sizes[0])
        return self._mats

    # ---- Fourier part -------------------------------------------------------------
    def fourier_forward(self, u):
        out = np.asarray(u)
        axes = self.fourier_axes
        for d in reversed(axes):
            if self.kinds[d] == "r2c":
                out = fourier.r2c_forward(out, d)
            else:
                out = fourier.c2c_forward(out.astype(np.complex128), d)
        return out

    def fourier_backward(self, u_hat):
        out = np.asarray(u_hat, dtype=np.complex128)
        for d in self.fourier_axes:
            if self.kinds[d] == "r2c":
                out = fourier.c2r_backward(out, self.sizes[d], d)
            else:
                out = fourier.c2c_backward(out, d)
        return out

    # ---- Shen part ------------------------------------------------------------------
    def _shen_scalar(self, g):
        kind, N = self.kinds[0], self.sizes[0]
        x, w = quadrature.points(kind, N)
        phi = quadrature.basis_values(kind, N, x)              # (N, nb)
        nb = phi.shape[1]
        s = np.tensordot((phi * w[:, None]).T, g, axes=([1], [0]))
        out = np.zeros((N,) + np.shape(g)[1:], dtype=s.dtype)
        out[:nb] = s
        return out

    def _shen_backward(self, c):
        kind, N = self.kinds[0], self.sizes[0]
        x, _ = quadrature.points(kind, N)
        phi = quadrature.basis_values(kind, N, x)
        nb = phi.shape[1]
        return np.tensordot(phi, np.asarray(c)[:nb], axes=([1], [0]))

    # ---- public -----------------------------------------------------------------------
    def scalar_product(self, f):
        """S(F(f)): Fourier transforms, then the Shen scalar product on axis 0."""
        g = self.fourier_forward(f)
        return self._shen_scalar(g) if self.has_cheb else g

    def forward(self, u):
        """u_hat = B^{-1} S(F(u)) (projection; Sec. 3.4.2)."""
        s = self.scalar_product(u)
        if not self.has_cheb:
            return s
        mats = self.matrices()
        return galerkin.solve_columns(self.kinds[0], self.sizes[0], s,
                                      np.zeros(s.shape[1:]), lambda k2: mats["B"])

    def backward(self, u_hat):
        g = self._shen_backward(u_hat) if self.has_cheb else np.asarray(u_hat)
        out = self.fourier_backward(g) if self.fourier_axes else g
        return out.real if self.real else out

    def helmholtz(self, a, b, f_tilde):
        """Solve the weak form of a lap(u) + b u = f, given S(F(f)) (Eq. laplace).

        Neumann basis: a column with b - a kappa2 = 0 (pure Poisson in the constant Fourier mode)
        determines u only up to a constant; there u_hat_0 = 0 and the phi_0 equation is dropped.
        """
        mats = self.matrices()
        singular = (lambda k2: b - a * k2 == 0.0) if self.kinds[0] == "neumann" else None
        return galerkin.solve_columns(self.kinds[0], self.sizes[0], f_tilde, self.kappa2(),
                                      lambda k2: galerkin.helmholtz_matrix(mats, a, b, k2), singular)

    def biharmonic(self, a, b, c, f_tilde):
        """Solve the weak form of a lap^2(u) + b lap(u) + c u = f, given S(F(f))."""
        mats = self.matrices()
        return galerkin.solve_columns(self.kinds[0], self.sizes[0], f_tilde, self.kappa2(),
                                      lambda k2: galerkin.biharmonic_matrix(mats, a, b, c, k2))

    # ---- derivatives (Sec. 5) ------------------------------------------------------------
    def project_dx(self, u_hat, axis, order, target=None):
        """project(Dx(u, axis, order), W0) of Sec. 5 for the Function with coefficients u_hat.

        W0 is this space with axis 0 replaced by `target` (default: the regular basis of its
        family, T_k or L_k; a Shen basis of the same family may be named instead, e.g.
        "dirichlet" or "biharmonic"); W0 is the space itself when every axis is a Fourier axis.
        The projection onto W0 is the forward transform of Sec. 3.4.2 applied to the
        derivative, written with Galerkin matrices:
          Chebyshev axis    B0^{-1} C u_hat, with C[k, l] = (d^m phi_l / dx^m, psi_k)_w^N and
                            W0's mass matrix B0[k, j] = (psi_j, psi_k)_w^N (psi the basis of
                            W0 along axis 0), both by Gauss quadrature (the projection of the
                            basis functions alone, m = 0, when the derivative is along a
                            Fourier axis);
          Fourier axis d    the Fourier inner products of Sec. 3.4.1 give the factor
                            (i k)^m, k = 2 pi l / L_d with the stored wavenumber l (FFT order;
                            an R2C axis keeps l = 0..M/2).
        Rows of u_hat past the basis size are ignored.  Returns the coefficients in W0's
        spectral layout (all N rows along axis 0, rows past W0's basis size zero).
        """
        u_hat = np.asarray(u_hat)
        ndim = len(self.kinds)
        assert 0 <= axis < ndim and order >= 0
        out = u_hat.astype(np.complex128 if np.iscomplexobj(u_hat) else np.float64)
        if self.has_cheb:
            kind, N = self.kinds[0], self.sizes[0]
            m0 = order if axis == 0 else 0
            tk = quadrature.regular_kind(kind) if target is None else target
            assert quadrature.family(tk) == quadrature.family(kind), "target must be of the same family"
            x, w = quadrature.points(kind, N)
            T = quadrature.basis_values(tk, N, x)                 # psi_k at x_j, (N, nt)
            V = quadrature.basis_values(kind, N, x, deriv=m0)     # phi_l^(m0)(x_j), (N, nb)
            nb, nt = V.shape[1], T.shape[1]
            Tw = T * w[:, None]
            C = Tw.T @ V
            B0 = Tw.T @ T
            res = np.tensordot(np.linalg.solve(B0, C), out[:nb], axes=([1], [0]))
            out = np.zeros((N,) + res.shape[1:], dtype=res.dtype)
            out[:nt] = res
        if not (self.has_cheb and axis == 0):
            M = self.sizes[axis]
            L = self.domains[axis][1] - self.domains[axis][0]
            k = fourier.wavenumbers(M, r2c=self.kinds[axis] == "r2c") * (2 * np.pi / L)
            view = [1] * ndim
            view[axis] = -1
            out = out * ((1j * k) ** order).reshape(view)
        return out
