"""Plain FP64 CPU oracle for the spectral Galerkin hot path (test infrastructure).

This package is test infrastructure only: the tests, the ``smoke()`` check and the
CPU-baseline leg of ``bench.py`` may import it; the product library never does.
It shares no code with the CUDA path.  Every transform here is a dense O(N^2)
quadrature or DFT sum, every Galerkin matrix is assembled by brute-force
Gauss-Chebyshev quadrature, and every solve is a dense LU (``numpy.linalg.solve``),
so that each function can be checked against the paper by eye.

Modules
  quadrature      Chebyshev-Gauss points/weights and basis values (Sec. 3.4.2).
  fourier         dense Fourier transforms and wavenumbers (Sec. 3.4.1).
  galerkin        mass / stiffness / bi-harmonic matrices by quadrature (Sec. 3.4.2, Sec. 4).
  space           tensor-product scalar product, forward, backward and solves (Sec. 4),
                  projected derivatives (Sec. 5).
  ginzburg_landau padded nonlinear term and RK4 steppers (Sec. 6).
  closure_cnn     periodic 3x3 convolution network, forward and backward (FP64).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
value the paper prints, a closed form, or an invariant, except the learned
closure's trained weights (parity unpinned: they depend on stochastic training);
the network's forward/backward arithmetic itself is pinned by finite differences.
"""
