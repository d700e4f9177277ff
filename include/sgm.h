/*
 * sgm.h - C ABI of libsgm, a GB300 (sm_103a) implementation of the data-parallel
 * hot path of the spectral Galerkin method of Mortensen, "Shenfun - automating the
 * spectral Galerkin method" (arXiv 1708.03188).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every data pointer is a DEVICE pointer owned by the caller (for example a torch
 *    tensor's data_ptr()), C-contiguous, and 16-byte aligned.  The library never frees
 *    caller memory.  Objects created by the library (spaces, Ginzburg-Landau steppers)
 *    own their device tables and workspaces and release them in the matching destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls are asynchronous on that stream; errors raised by a kernel after launch
 *    are reported by a later call or by the caller's synchronisation.
 *  - Every call returns an int status: SGM_OK (0) or a negative SGM_ERR_* code.
 *    sgm_last_error() returns a thread-local message for the last failure.  Nothing
 *    crosses the ABI as a C++ exception.
 *  - Input and output arrays must not overlap (SGM_ERR_ALIAS), except where a call
 *    says it works in place.
 *
 * Data layout (Sec. 4 of the paper; the default axis order of its TensorProductSpace)
 * -------------------------------------------------------------------------------
 *  A space has ndim axes.  Either axis 0 is a polynomial axis (SGM_CHEBYSHEV,
 *  SGM_SHEN_DIRICHLET, SGM_SHEN_BIHARMONIC, or the Legendre bases SGM_LEGENDRE*) and axes 1..
 *  are Fourier axes, or all axes are Fourier axes.  Only the last axis may be SGM_FOURIER_R2C.
 *  Physical arrays have shape (n[0], ..., n[ndim-1]); they are real when the last
 *  axis is R2C or the space is one Chebyshev axis alone, complex otherwise.
 *  Spectral arrays are complex (interleaved re, im) of shape (n[0], ..., m) with
 *  m = n[ndim-1]/2 + 1 for an R2C last axis, else n[ndim-1]; a 1-D Chebyshev
 *  space has a real spectral array of length n[0].  Along the Chebyshev axis all n[0]
 *  rows are stored; rows past the basis size (the index sets l^D = 0..N-3 of
 *  Sec. 3.4.2 and l^B = 0..N-5 of Sec. 4) are written as zero.  Fourier axes are in
 *  FFT order (l = 0, 1, ..., -2, -1).
 *  Precision SGM_F32: float / complex64 arrays, FFTs and DCTs in FP32, every
 *  Helmholtz, biharmonic and mass-matrix elimination in FP64 (inputs widened,
 *  results rounded once).  SGM_F64: double / complex128 arrays, all arithmetic FP64.
 *
 * Normalisation (Sec. 3.4.1 and Sec. 3.4.2 of the paper)
 * -----------------------------------------------------
 *  Fourier forward:  u_hat_l = (1/M) sum_j u_j exp(-i l X_j), X_j = 2 pi j / M
 *  Fourier backward: u_j = sum_l u_hat_l exp(i l X_j)
 *  Shen scalar product on axis 0: S_k(u) = (u, phi_k)_w^N = (pi/N) sum_j u(x_j) phi_k(x_j),
 *  x_j = cos((2j+1) pi / (2N)).  The 2 pi (or domain length) factors of the Fourier
 *  inner products are divided out of both sides of every weak form.
 */
#ifndef SGM_H
#define SGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SGM_OK 0
#define SGM_ERR_NULL -1        /* a required pointer is NULL */
#define SGM_ERR_SIZE -2        /* unsupported size, dimension or basis combination */
#define SGM_ERR_ARG -3         /* invalid scalar argument */
#define SGM_ERR_ALIAS -4       /* input and output overlap */
#define SGM_ERR_ALIGN -5       /* pointer not 16-byte aligned */
#define SGM_ERR_CUDA -6        /* a CUDA runtime call failed (message in sgm_last_error) */
#define SGM_ERR_ALLOC -7       /* device or host allocation failed */
#define SGM_ERR_STATE -8       /* object used after destroy or with a mismatched kind */

/* basis kinds (Sec. 3.1 of the paper, the bases of shenfun.chebyshev and shenfun.fourier) */
#define SGM_CHEBYSHEV 0          /* regular T_k, k = 0..N-1 */
#define SGM_SHEN_DIRICHLET 1     /* T_k - T_{k+2}, k = 0..N-3 (Eq. chebdirichlet) */
#define SGM_SHEN_BIHARMONIC 2    /* T_k - 2(k+2)/(k+3) T_{k+2} + (k+1)/(k+3) T_{k+4}, k = 0..N-5 (Eq. chebbiharmonic) */
#define SGM_FOURIER_C2C 3        /* exp(i l x), complex data */
#define SGM_FOURIER_R2C 4        /* exp(i l x), real data, l = 0..M/2 stored (last axis only) */
/* Legendre bases (Sec. 3.1; Eq. legdirichlet; Eq. legbiharmonic with the factor L_{k+4} of its last
 * term, which the printed formula lacks and phi(+-1) = phi'(+-1) = 0 requires), axis 0 only,
 * 2 <= N <= 1024, on the Legendre-Gauss points in descending order (weight 1).  Their
 * transforms are dense O(N^2) sums (no fast transform is known, Sec. 3.4.2); their Helmholtz and
 * biharmonic systems are banded within a parity after integration by parts. */
#define SGM_LEGENDRE 5             /* L_k, k = 0..N-1 */
#define SGM_LEGENDRE_DIRICHLET 6   /* L_k - L_{k+2}, k = 0..N-3 */
#define SGM_LEGENDRE_BIHARMONIC 7  /* L_k - 2(2k+5)/(2k+7) L_{k+2} + (2k+3)/(2k+7) L_{k+4}, k = 0..N-5 */
/* Shen Neumann basis (Sec. 3.1 lists ShenNeumannBasis without its formula; this is the
 * combination with phi_k'(+-1) = 0), axis 0 only, N >= 4.  Its Helmholtz solve (sgm_helmholtz_solve,
 * sgm_helmholtz) handles a Fourier column whose system has no zeroth-order term (b - a kappa2
 * evaluates to exactly 0, e.g. the constant column of a Poisson problem) by setting u_hat_0 = 0
 * and dropping the equation of phi_0: u is then fixed up to the constant it cannot see. */
#define SGM_SHEN_NEUMANN 8         /* T_k - (k/(k+2))^2 T_{k+2}, k = 0..N-3 */

/* precision */
#define SGM_F32 1                /* FP32 transforms, FP64 eliminations */
#define SGM_F64 2                /* FP64 everywhere */
/* Chebyshev-axis method, or-ed into the precision of an SGM_F32 space (see sgm_space_create) */
#define SGM_CHEB_TC 0x10         /* dense BF16x3 tensor-core contraction (N <= 128) */
#define SGM_CHEB_AUTO 0x20       /* time both methods at creation and keep the faster */

/* shape selectors for sgm_space_shape */
#define SGM_PHYSICAL 0
#define SGM_SPECTRAL 1

typedef struct sgm_space sgm_space;

/* Thread-local description of the last failure on the calling thread. */
const char* sgm_last_error(void);
/* Static text for a status code. */
const char* sgm_status_string(int status);

/*
 * Create a tensor-product space (the TensorProductSpace of Sec. 4; bases of Sec. 3.1).
 *   out        receives the new space.
 *   ndim       1..3.
 *   kinds      ndim basis kinds (see above), in the order of the array axes.  The canonical
 *              order puts the Chebyshev or Legendre axis first and the R2C axis last; any other
 *              order (the axes option of Sec. 4, e.g. TensorProductSpace((K1, K0), axes=(1, 0))
 *              with the Dirichlet basis along the second axis) gives a view of the canonical
 *              space whose arrays are axis permutations of the canonical ones: every call
 *              permutes its input into a canonical workspace, runs the canonical call and
 *              permutes the result back (two extra passes over the data).  At most one
 *              polynomial and one R2C axis.  Axis arguments (sgm_project_dx, sgm_project) and
 *              shapes (sgm_space_shape) follow the array order.
 *   n          ndim sizes: quadrature points per axis (N >= 4 for Dirichlet, 6 <= N <= 2048
 *              for biharmonic, N <= 1024 for the Legendre bases; Fourier sizes >= 1).  Every
 *              size <= 4096.
 *   domain     2*ndim doubles (lo, hi) per axis, or NULL for [-1,1] on a Chebyshev axis
 *              and [0, 2 pi) on a Fourier axis.  A Fourier axis of length L = hi - lo is
 *              mapped onto [0, 2 pi), so its derivatives scale by 2 pi / L (Sec. 6).
 *              A Chebyshev or Legendre axis must keep [-1, 1].
 *   precision  SGM_F32 or SGM_F64.  An SGM_F32 space with a Chebyshev or Legendre axis of
 *              N <= 128 points may add one axis-0 method flag (for a Legendre axis the
 *              alternative to the tensor cores is its dense CUDA-core product, not an FFT):
 *                SGM_CHEB_TC    the Chebyshev-axis scalar product, forward T_k transform and
 *                               backward transform run as one dense N x N contraction per
 *                               column on the tensor cores (tcgen05, BF16x3 split products,
 *                               FP32 accumulation) instead of the DCT-via-FFT kernels.
 *                               Error: each product carries at most ~3 * 2^-16 relative
 *                               error (the dropped lo*lo product and the BF16 rounding of
 *                               the lo parts), ~2^-18 relative L2 per contraction in
 *                               practice; SGM_ERR_SIZE if N > 128.
 *                SGM_CHEB_AUTO  time both methods on this space at creation (on a private
 *                               stream, device-synchronising) and keep the faster; N > 128
 *                               keeps the FFT method.
 *              The flags are an SGM_ERR_ARG for SGM_F64 spaces.
 * Allocates device tables and workspace on the current device (freed by destroy).  A 3-D space
 * whose axis 0 is SGM_SHEN_DIRICHLET or SGM_SHEN_BIHARMONIC also holds two factorisation slots
 * (see the solves below): 2 x (n[0]/2 + 1) x 4 (Dirichlet) or 7 (biharmonic) doubles per pair of
 * Fourier columns +-l1 and parity, e.g. 2 x 237 MB for the biharmonic basis on a 256^3 box.
 */
int sgm_space_create(sgm_space** out, int ndim, const int* kinds, const int64_t* n,
                     const double* domain, int precision);
/* Release a space and everything it owns.  NULL is accepted and ignored. */
int sgm_space_destroy(sgm_space* space);
/* Write the ndim extents of the PHYSICAL or SPECTRAL array into shape_out. */
int sgm_space_shape(const sgm_space* space, int which, int64_t* shape_out);
/*
 * Measurement hook (no counterpart in the paper): events (cudaEvent_t passed as void*, owned by the
 * caller) that the physical-to-physical solves of this space (sgm_helmholtz, sgm_biharmonic) record
 * on the caller's stream right before and right after their elimination kernel, so that a caller
 * can time that kernel inside a longer sequence of work.  Both NULL clears them; one NULL is
 * SGM_ERR_ARG.  The events are recorded by every later solve until cleared.
 */
int sgm_space_solve_events(sgm_space* space, void* begin, void* end);
/* Chebyshev-axis method in use: *method = 0 (DCT via FFT), 1 (tensor-core contraction). */
int sgm_space_cheb_method(const sgm_space* space, int* method);
/*
 * Number of bounded waits inside tensor-core kernels (Chebyshev contraction, 32 -> 32 convolution
 * layers) on the current device that gave up
 * (each wait gives up after ~1 s; the kernel then skips its result and returns).  Reads a
 * device counter synchronously; reset != 0 also zeroes it.  A non-zero count means the
 * results of those launches are invalid.
 */
int sgm_tc_wait_timeouts(int* count, int reset);

/*
 * Scalar product S(F(f)) (the `inner(v, f)` of Sec. 3.4.2 and the right-hand side
 * formula of Sec. 4): Fourier forward transforms (R2C on the last axis, then C2C axes
 * from last to first), then the Shen scalar product on axis 0 computed as a DCT-II
 * (via an FFT) with the basis stencil applied to the Chebyshev moments.
 *   f        physical array;  f_tilde  spectral array (output).
 * Pure Fourier spaces return the Fourier coefficients.
 */
int sgm_scalar_product(sgm_space* space, const void* f, void* f_tilde, void* stream);

/*
 * Forward transform u_hat = B^{-1} S(F(u)) (the projection T of Sec. 3.4.2): the scalar
 * product followed by the mass-matrix solve along axis 0 in FP64.
 */
int sgm_forward(sgm_space* space, const void* u, void* u_hat, void* stream);

/*
 * Backward transform (Eq. fast_shen, then the inverse Fourier transforms): the basis
 * stencil turns Shen coefficients into Chebyshev coefficients, a DCT-III (via an FFT)
 * evaluates them at the Gauss points, then inverse C2C and C2R transforms.
 */
int sgm_backward(sgm_space* space, const void* u_hat, void* u, void* stream);

/*
 * Helmholtz/Poisson solve on a Shen-Dirichlet space (Eq. laplace; the Helmholtz solver of
 * Sec. 4): for every Fourier column with squared wavenumber kappa^2 solve, in FP64,
 *     (a (A - kappa^2 B) + b B) u_hat = f_tilde,
 * the weak form of  a lap(u) + b u = f.  A is the stiffness matrix (phi_l'', phi_m)_w and
 * B the mass matrix of Sec. 3.4.2.  Poisson -lap(u) = f is a = -1, b = 0.
 *   f_tilde  spectral right-hand side (S(F(f)));  u_hat  spectral solution.
 * Works in place (f_tilde == u_hat).  Requires axis 0 = SGM_SHEN_DIRICHLET or
 * SGM_LEGENDRE_DIRICHLET (whose A is diagonal, -(4k+6), and B tridiagonal within a parity).
 * a = b = 0, or a system with a zero pivot, gives SGM_ERR_ARG / non-finite output.
 */
/*
 * Factorisation slots (3-D spaces with a Shen Dirichlet or biharmonic axis 0; the paper builds its
 * Helmholtz and Biharmonic solvers once from their matrices and applies them to many right-hand
 * sides, Sec. 4).  The FP64 factorisation of every column system depends only on the operator
 * (a, b, c) and kappa^2.  Such a space keeps the factorisations of the last two operators it
 * solved with (the mass solve of sgm_forward counts as one), per column layout (spectral arrays,
 * or the padded intermediates of the physical-to-physical solves).  A solve with an operator in a
 * slot replays only the right-hand-side recurrences; a solve with another operator first computes
 * its factorisation into the least recently used slot, on the call's stream (the first solve with
 * new coefficients costs about two solves).  Inside a stream capture the solves neither read nor
 * fill the slots: the captured graph runs kernels that factor as they solve, so it stays valid
 * whatever later calls store in the slots.  Results are those of the same FP64 arithmetic either
 * way, up to the order of the back substitution's sums.  Calls on one space must not overlap on the
 * GPU (they share its workspaces and slots) and must come from one host thread at a time.
 */
int sgm_helmholtz_solve(sgm_space* space, double a, double b, const void* f_tilde,
                        void* u_hat, void* stream);

/*
 * Biharmonic solve on a Shen-biharmonic space (Sec. 4, the Biharmonic solver): for every
 * Fourier column solve, in FP64,
 *     (a (S - 2 kappa^2 A + kappa^4 B) + b (A - kappa^2 B) + c B) u_hat = f_tilde,
 * the weak form of  a lap^2(u) + b lap(u) + c u = f,  S = (phi_l'''', phi_m)_w.
 * The paper's problem lap^2(u) = f is a = 1, b = c = 0.  Works in place.
 * Requires axis 0 = SGM_SHEN_BIHARMONIC or SGM_LEGENDRE_BIHARMONIC (whose S is diagonal, A
 * tridiagonal and B pentadiagonal within a parity).
 */
int sgm_biharmonic_solve(sgm_space* space, double a, double b, double c, const void* f_tilde,
                         void* u_hat, void* stream);

/*
 * Physical-to-physical Helmholtz solve: u = backward(solve(scalar_product(f))), the whole
 * pipeline of the paper's Fig. poisson2D in one call.  f and u are physical arrays.
 */
int sgm_helmholtz(sgm_space* space, double a, double b, const void* f, void* u, void* stream);
/* Physical-to-physical biharmonic solve (scalar product, biharmonic solve, backward). */
int sgm_biharmonic(sgm_space* space, double a, double b, double c, const void* f, void* u,
                   void* stream);

/*
 * Projected derivative, project(Dx(u, axis, order), W0) of Sec. 5: the coefficients in W0 of
 * the order-th partial derivative along `axis` of the Function u whose coefficients in this
 * space are u_hat.  W0 is this space with axis 0 replaced by SGM_CHEBYSHEV, or by SGM_LEGENDRE for
 * the Legendre bases (same sizes, domain and precision); when every axis is a Fourier axis, W0 is
 * this space itself.  Legendre bases use the Legendre derivative recurrence
 * b_r / (2r+1) = b_{r+2} / (2r+5) + a_{r+1} in place of the Chebyshev one below.  The projection
 * is exact (every polynomial degree stays below N), so du_hat holds the Chebyshev
 * coefficients of the derivative: the basis stencil of the space (Eq. fast_shen) maps u_hat
 * to Chebyshev coefficients, then
 *   axis 0         the Chebyshev derivative recurrence  c_k b_k = b_{k+2} + 2(k+1) a_{k+1}
 *                  (c_0 = 2, c_k = 1 otherwise), applied `order` times;
 *   Fourier axis   the factor (i k)^order, k = 2 pi l / L with the stored wavenumber l
 *                  (FFT order; an even-length C2C axis stores the Nyquist mode as l = -M/2, an
 *                  R2C axis as l = +M/2).
 *   u_hat   spectral array of this space (rows past the basis size are ignored);
 *   du_hat  spectral array of the same shape and type (output, all N rows written).
 * 0 <= axis < ndim and 0 <= order <= 4, else SGM_ERR_ARG.  Out of place only (SGM_ERR_ALIAS).
 * SGM_F32 spaces compute in FP32 pairs (hi + lo, error-free products and sums) and round
 * once; SGM_F64 spaces compute in FP64.
 */
int sgm_project_dx(sgm_space* space, int axis, int order, const void* u_hat, void* du_hat,
                   void* stream);

/*
 * Projection onto another space, project(Dx(u, axis, order), W) of Sec. 5 with any target W
 * that differs from this space at most in the basis of axis 0: the regular basis of the same
 * family (then identical to sgm_project_dx) or a Shen basis of that family (SGM_SHEN_DIRICHLET,
 * SGM_SHEN_BIHARMONIC, or the Legendre ones).  For a Shen target the result is the Galerkin
 * projection: the coefficients c in W with (sum_j c_j psi_j, psi_k)_w = (d^m u, psi_k)_w for every
 * basis function psi_k of W, computed from the derivative's regular coefficients d (as
 * sgm_project_dx) by the exact scalar products S_k = w_k d_k + beta_k w_{k+2} d_{k+2} + gamma_k
 * w_{k+4} d_{k+4} (w_k = pi c_k / 2 Chebyshev, 2 / (2k+1) Legendre; beta, gamma the target's
 * stencil) and the FP64 mass solve of the forward transform (Sec. 3.4.2).
 *   target   a live space of the same ndim, sizes, domains and precision (SGM_ERR_STATE
 *            otherwise); Fourier-only spaces: target has the same kinds.
 *   u_hat    spectral array of `space`; out_hat: spectral array of `target` (all N rows
 *            written, rows past the target basis zero).  Out of place (SGM_ERR_ALIAS).
 * Uses the workspaces of both spaces: calls on either space must not overlap on the GPU.
 */
int sgm_project(sgm_space* space, int axis, int order, const void* u_hat, sgm_space* target, void* out_hat,
                void* stream);

/* ---- complex Ginzburg-Landau equation (Sec. 6 of the paper) ------------------------------- */
#define SGM_GL_RK4 0      /* explicit classical RK4, the paper's time loop */
#define SGM_GL_IFRK4 1    /* classical RK4 on exp(-L t) u_hat (linear part integrated exactly) */

typedef struct sgm_gl sgm_gl;

/*
 * Create a stepper for  u_t = u + (1 + i beta) lap(u) - (1 + i gamma) |u|^2 u  on the space
 * (a square M x M SGM_FOURIER_C2C x SGM_FOURIER_C2C space; M in {32, 64, ..., 1024}; equal
 * domain lengths, e.g. [-50, 50]^2 as in Sec. 6).  The paper's equation is beta = 0,
 * gamma = 1.5.  In Fourier space du_hat/dt = L(k) u_hat - N(u_hat), L(k) = 1 - (1 + i beta)|k|^2,
 * with the nonlinear term N evaluated with the padded transforms of Sec. 6: padding must be
 * 1.5 (coefficients copied to an (3M/2)^2 array at the same wavenumbers, zero elsewhere;
 * backward transform unscaled; forward transform with 1/(3M/2) per axis, truncated).
 * dt > 0; scheme SGM_GL_RK4 or SGM_GL_IFRK4.  Precision follows the space (SGM_F32: complex64
 * state and FP32 arithmetic; SGM_F64: complex128 and FP64).  The space may be destroyed
 * after this call; the stepper owns its workspaces and tables.
 */
int sgm_gl_create(sgm_gl** out, const sgm_space* space, double padding, double beta, double gamma,
                  double dt, int scheme);
int sgm_gl_destroy(sgm_gl* gl);
/* rhs = L(k) u_hat - N(u_hat) for a spectral M x M state u_hat (FFT order on both axes). */
int sgm_gl_rhs(sgm_gl* gl, const void* u_hat, void* rhs, void* stream);
/* Advance u_hat (in place) by nsteps time steps of the stepper's scheme. */
int sgm_gl_step(sgm_gl* gl, void* u_hat, int nsteps, void* stream);

/* ---- batched independent 1-D Helmholtz problems ------------------------------------------- */
typedef struct sgm_batch sgm_batch;

/*
 * Describe a batch of nprob independent problems  u_p'' - alpha_p u_p = f_p  on [-1, 1] with
 * u_p(+-1) = 0, problem p on its own Chebyshev-Gauss grid of n[p] points (4 <= n[p] <= 4096),
 * discretised with the Shen-Dirichlet basis (Sec. 3.4.2; the weak form of sgm_helmholtz_solve
 * with a = 1, b = -alpha_p, kappa = 0).  precision SGM_F32 (FP32 transforms, FP64
 * eliminations) or SGM_F64.  Builds the size-sorted problem table, per-size FFT plans and
 * twiddles and the FP64 work buffers on the current device.  nprob may be 0 (n and alpha
 * are then ignored) for a batch of 2-D problems only (sgm_batch_add_2d).
 */
int sgm_batch_create(sgm_batch** out, int nprob, const int64_t* n, const double* alpha, int precision);
/* or-ed into the precision of sgm_batch_create: keep the default plan (Bluestein above a largest
 * prime factor of 32) instead of autotuning it (see sgm_batch_info) */
#define SGM_BATCH_FIXED_PLAN 0x40
int sgm_batch_destroy(sgm_batch* batch);
/* Element offsets of the problems in the packed arrays: offsets[p] = n[0] + ... + n[p-1], nprob+1 entries. */
int sgm_batch_offsets(const sgm_batch* batch, int64_t* offsets);
/*
 * Solve every problem: f and u are packed real arrays (float or double) of sum(n) values,
 * problem p at offsets[p] (the samples at x_j = cos((2j+1) pi / (2 n[p])).  Three kernel
 * launches on `stream`: DCT-II + stencil per problem, the FP64 eliminations (32 problems per
 * warp), stencil + DCT-III per problem.  f and u must not overlap.
 */
int sgm_batch_helmholtz(sgm_batch* batch, const void* f, void* u, void* stream);
/*
 * Plan chosen at creation.  A size N whose largest prime factor exceeds *bluestein_prime runs its
 * DFT as a Bluestein convolution of a power-of-two length; the others run their mixed-radix plan.
 * The threshold is autotuned: sgm_batch_create times the whole batch on zero input for each of
 * 16, 32, 64 and "never" (*bluestein_prime = 0) and keeps the fastest.  *n_bluestein counts the
 * problems on the Bluestein path.
 */
int sgm_batch_info(const sgm_batch* batch, int* bluestein_prime, int* n_bluestein);
/*
 * Add nprob independent 2-D problems  a lap(u_q) + b u_q = f_q  on [-1, 1] x [0, 2 pi), each
 * on its own Shen-Dirichlet x R2C Fourier space (the 2-D Poisson problem of Sec. 4, solved as
 * sgm_helmholtz does: scalar product, per-wavenumber FP64 elimination, backward transform).
 * sizes: 2 per problem (N >= 4 Chebyshev points, M >= 2 Fourier points, both <= 4096).  One
 * space per problem is created on the current device, with SGM_CHEB_AUTO for SGM_F32 batches
 * (the Chebyshev-axis method of each size is chosen by timing).  a, b as in sgm_helmholtz,
 * common to the problems added by this call.  May be called once per batch, before the first
 * sgm_batch_run.
 */
int sgm_batch_add_2d(sgm_batch* batch, int nprob, const int64_t* sizes, double a, double b);
/*
 * Element offsets of the 2-D problems in their packed real arrays (nprob + 1 entries): problem
 * q's row-major N x M samples start at offsets[q], a multiple of 4, so every problem is 16-byte
 * aligned; offsets[nprob] is the total length.
 */
int sgm_batch_offsets_2d(const sgm_batch* batch, int64_t* offsets);
/*
 * Solve every problem of the batch (1-D: f1 -> u1 as sgm_batch_helmholtz; 2-D: f2 -> u2) as ONE
 * CUDA graph launch on `stream`.  The first call, and any call whose four pointers differ from
 * those of the captured graph, runs each problem once eagerly (so that every lazily built
 * table exists), then captures the graph on internal streams: the 1-D kernels on one branch and
 * the 2-D problems spread over up to 64 concurrent branches, longest first; that call
 * synchronises the device.  Later calls only launch the graph (asynchronous).  f1/u1 may be NULL
 * when the batch has no 1-D problems, f2/u2 when it has no 2-D problems.  Calls on one batch
 * must not overlap.
 */
int sgm_batch_run(sgm_batch* batch, const void* f1, void* u1, const void* f2, void* u2, void* stream);

/* ---- learned closure kernels (no counterpart in the paper) -----------------------------------
 * A periodic 3x3 convolution layer is the circular cross-correlation
 *   y[b,o,i,j] = bias[o] + sum_{c,p,q} W[o,c,p,q] x[b,c,(i+p-1) mod H,(j+q-1) mod W],  p, q = 0..2,
 * with x, W, y stored as BF16 (W laid out [Cout][Cin][3][3]; the input layer's x may be FP32),
 * bias and every accumulation FP32.
 * Supported channel pairs (Cin, Cout): (2, 32), (32, 32), (32, 2); H and W multiples of 16;
 * arrays [B][C][H][W], C-contiguous device memory. */
#define SGM_CONV_RELU 1      /* apply ReLU to the output */
#define SGM_CONV_OUT_F32 2   /* y is FP32 (else BF16) */
#define SGM_CONV_IN_F32 4    /* x is FP32 (else BF16); the 2-channel input layer only */
/* y = conv(x), options in `flags` (SGM_CONV_*). */
int sgm_conv3x3_forward(const void* x, const void* w, const float* bias, void* y, int B, int Cin, int Cout,
                        int H, int W, int flags, void* stream);
/* gx = d(sum gy * y)/dx for one layer (FP32 gy, gx); when mask (the BF16 layer input, itself a
 * ReLU output) is non-NULL, gx is zeroed where mask <= 0 (the derivative of that ReLU). */
int sgm_conv3x3_backward_data(const float* gy, const void* w, const void* mask, float* gx, int B, int Cin,
                              int Cout, int H, int W, void* stream);
/* gw += d(sum gy * y)/dW, gb += d(sum gy * y)/dbias (FP32, accumulated with atomics); x as in
 * the forward call (flags: SGM_CONV_IN_F32). */
int sgm_conv3x3_backward_weights(const float* gy, const void* x, float* gw, float* gb, int B, int Cin,
                                 int Cout, int H, int W, int flags, void* stream);
/* One AdamW step on n FP32 master values w (moments m, v; decoupled weight decay); when w_bf16
 * is non-NULL the updated values are also written there in BF16.  step >= 1 (bias correction). */
int sgm_adamw_step(float* w, void* w_bf16, const float* g, float* m, float* v, int64_t n, float lr, float beta1,
                   float beta2, float eps, float weight_decay, int step, void* stream);
/* grad = 2 (out - target) / n and *loss += sum (out - target)^2 / n (FP32; *loss accumulated). */
int sgm_mse_grad(const float* out, const float* target, float* grad, float* loss, int64_t n, void* stream);
/* Keep the wavenumbers of an Mc x Mc grid from B complex64 Mf x Mf spectral arrays (FFT order). */
int sgm_spectral_truncate(const void* src, int Mf, void* dst, int Mc, int B, void* stream);
/*
 * Training batch of the learned closure (no counterpart in the paper: a data transform built
 * from the symmetries of the Ginzburg-Landau equation, Sec. 6 - the equation is invariant under
 * a global phase u -> exp(i theta) u, periodic translations, the transposition of the square
 * grid and the reflections x -> -x, y -> -y).  For b < B, with k = idx[b], the complex64 fields
 * u[k] and d[k] of the pools u, d ([n][M][M], device) are multiplied by phase[b] (B complex64
 * values, device), rolled by (sx, sy) along axes (0, 1) (value at (i, j) moves to
 * ((i + sx) mod M, (j + sy) mod M)), transposed when SGM_AUG_TRANSPOSE, then reflected along
 * axis 0 (SGM_AUG_FLIP0: index i -> (M - i) mod M) and axis 1 (SGM_AUG_FLIP1), and written as
 * FP32 channels xu[b][0] = su Re, xu[b][1] = su Im ([B][2][M][M], device), and xd from d with sd.
 * idx: B int32 (device), each in [0, n); an entry outside writes zeros for that sample.
 * sx, sy >= 0, flags a combination of SGM_AUG_* (SGM_ERR_ARG otherwise).
 */
#define SGM_AUG_TRANSPOSE 1
#define SGM_AUG_FLIP0 2
#define SGM_AUG_FLIP1 4
int sgm_augment_pack(const void* u, const void* d, int n, int M, const int* idx, const void* phase, int B, int sx,
                     int sy, int flags, float su, float sd, float* xu, float* xd, void* stream);
/* x[b,0] = scale Re u[b], x[b,1] = scale Im u[b] (complex64 -> BF16 channels, B x H x W fields). */
int sgm_pack_channels(const void* u, void* x, int B, int H, int W, float scale, void* stream);
/* u[b] += scale (d[b,0] + i d[b,1]) (FP32 channels added to complex64 fields). */
int sgm_unpack_add(const float* d, void* u, int B, int H, int W, float scale, void* stream);

/*
 * Fused multiply-add throughput probe (a measurement utility, no counterpart in the paper).
 * Launches blocks x threads threads, each running 8 independent FMA chains for `iters`
 * rounds in FP64 (precision SGM_F64) or FP32 (SGM_F32), and writes one value per thread to
 * the device array `sink` (blocks * threads doubles or floats).  *flops (host) receives the
 * flop count of the launch (2 per FMA), to be divided by the launch's event-timed duration.
 * threads: a multiple of 32 in 32..256; SGM_ERR_SIZE otherwise.
 */
int sgm_alu_probe(int precision, int blocks, int threads, int64_t iters, void* sink, double* flops, void* stream);

/*
 * Dirichlet Helmholtz solve that allocates nothing (no counterpart in the paper; it is an
 * interface choice of this library).
 *
 * For callers that must not allocate device memory themselves: programs whose device
 * memory belongs to one memory manager (a framework's caching allocator, or a fixed budget
 * reserved up front) and latency-critical loops that cannot afford the time or the possible
 * failure of cudaMalloc.  sgm_space_create allocates, so those callers cannot use the space
 * API; this entry point computes the same result as sgm_helmholtz_solve on a space built
 * from the same arguments, with no space object and no cudaMalloc/cudaFree.
 *   ndim, kinds, n, domain, precision   as for sgm_space_create; kinds[0] must be
 *                                       SGM_SHEN_DIRICHLET and 4 <= n[0] <= 2048.
 *   a, b, f_tilde, u_hat, stream        as for sgm_helmholtz_solve (in place allowed).
 *   domain may be NULL; when given, axis 0 must be [-1, 1].
 * Scratch: an 8 MiB array in the library's device memory, held until the process exits.
 * With CUDA's lazy module loading it is reserved on a device by the first call there, which
 * also looks up the array's device address (with that device current) and caches it.  Make
 * that first call before any stream capture, and before a fixed-budget caller claims the rest
 * of the device's memory (otherwise the first call can fail with SGM_ERR_CUDA).  The cached
 * address belongs to the primary context: do not call this entry point again after
 * cudaDeviceReset in the same process.  All calls share the array and it keeps the last
 * call's contents (nothing in it needs to start at zero); calls whose kernels overlap on the
 * GPU, e.g. on two streams, race on it, so serialise them.  Sizes past the limit return
 * SGM_ERR_SIZE.
 * Cost: the array bounds the number of threads to 8 MiB / (32 B (N/2 + 1)), i.e. 128-thread
 * CTAs: 15 at N = 256, 3 at N = 1024, 2 from N = 1364 and 1 at N = 2048, against one thread per
 * (column, parity) for sgm_helmholtz_solve.  Large N on many columns therefore runs on few SMs;
 * use this entry point where allocation is impossible, not for throughput at large N.
 */
int sgm_helmholtz_solve_noalloc(int ndim, const int* kinds, const int64_t* n, const double* domain,
                                int precision, double a, double b, const void* f_tilde, void* u_hat,
                                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SGM_H */
