"""ctypes binding of libsgm (include/sgm.h): argument marshalling only.

Every computation runs in the CUDA kernels of libsgm.so; this module checks tensor
shapes and dtypes, passes device pointers and the current CUDA stream, and turns
status codes into exceptions.  There is no CPU fallback: if libsgm.so is missing the
first call raises.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgm.so")

KINDS = {"chebyshev": 0, "dirichlet": 1, "biharmonic": 2, "c2c": 3, "r2c": 4,
         "legendre": 5, "legendre_dirichlet": 6, "legendre_biharmonic": 7, "neumann": 8}
POLYNOMIAL = ("chebyshev", "dirichlet", "biharmonic", "neumann", "legendre", "legendre_dirichlet",
              "legendre_biharmonic")
PRECISION = {"f32": 1, "f64": 2}
CHEB_METHOD = {"fft": 0, "tc": 0x10, "auto": 0x20}
_VP = ctypes.c_void_p
_D = ctypes.c_double

_SIGNATURES = {
    "sgm_last_error": (ctypes.c_char_p, []),
    "sgm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sgm_space_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_D), ctypes.c_int]),
    "sgm_space_destroy": (ctypes.c_int, [_VP]),
    "sgm_space_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "sgm_space_cheb_method": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "sgm_space_solve_events": (ctypes.c_int, [_VP, _VP, _VP]),
    "sgm_tc_wait_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "sgm_scalar_product": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sgm_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sgm_backward": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sgm_helmholtz_solve": (ctypes.c_int, [_VP, _D, _D, _VP, _VP, _VP]),
    "sgm_biharmonic_solve": (ctypes.c_int, [_VP, _D, _D, _D, _VP, _VP, _VP]),
    "sgm_helmholtz": (ctypes.c_int, [_VP, _D, _D, _VP, _VP, _VP]),
    "sgm_biharmonic": (ctypes.c_int, [_VP, _D, _D, _D, _VP, _VP, _VP]),
    "sgm_project_dx": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "sgm_project": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "sgm_gl_create": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, _D, _D, _D, _D, ctypes.c_int]),
    "sgm_gl_destroy": (ctypes.c_int, [_VP]),
    "sgm_gl_rhs": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sgm_gl_step": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "sgm_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(_D), ctypes.c_int]),
    "sgm_batch_destroy": (ctypes.c_int, [_VP]),
    "sgm_batch_offsets": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "sgm_batch_helmholtz": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sgm_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sgm_batch_add_2d": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _D, _D]),
    "sgm_batch_offsets_2d": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "sgm_batch_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sgm_conv3x3_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP]),
    "sgm_conv3x3_backward_data": (ctypes.c_int, [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 5 + [_VP]),
    "sgm_conv3x3_backward_weights": (ctypes.c_int, [_VP, _VP, _VP, _VP] + [ctypes.c_int] * 6 + [_VP]),
    "sgm_adamw_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int64] + [ctypes.c_float] * 5
                       + [ctypes.c_int, _VP]),
    "sgm_mse_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, _VP]),
    "sgm_spectral_truncate": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    "sgm_pack_channels": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, _VP]),
    "sgm_unpack_add": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, _VP]),
    "sgm_augment_pack": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float, _VP, _VP, _VP]),
    "sgm_alu_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _VP,
                                     ctypes.POINTER(_D), _VP]),
    "sgm_helmholtz_solve_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_D), ctypes.c_int,
                                                   _D, _D, _VP, _VP, _VP]),
}

_lib = None


class SgmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libsgm status {status}: {message}")
        self.status = status


def lib():
    """Load libsgm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1708_03188_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(status):
    if status != 0:
        raise SgmError(status, lib().sgm_last_error().decode())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return _VP(s.cuda_stream)


def _ptr(t):
    return _VP(t.data_ptr())


class Space:
    """Tensor-product space (one Chebyshev or Legendre axis + Fourier axes, or Fourier axes only).

    kinds: names from KINDS in the order of the array axes (the polynomial axis and the R2C axis
    may sit on any axis: the axes option of Sec. 4); sizes: quadrature points per axis; domain: [(lo, hi)] per
    axis or None; precision "f32" (FP32 transforms, FP64 solves) or "f64"; cheb (f32 only):
    "fft" (DCT via FFT), "tc" (dense BF16x3 tensor-core contraction, N <= 128) or "auto"
    (the faster of the two, timed at creation).
    """

    def __init__(self, kinds, sizes, domain=None, precision="f32", cheb="fft"):
        self.kinds = tuple(kinds)
        self.sizes = tuple(int(s) for s in sizes)
        self.precision = precision
        self.domain = domain
        nd = len(self.kinds)
        k = (ctypes.c_int * nd)(*[KINDS[x] for x in self.kinds])
        n = (ctypes.c_int64 * nd)(*self.sizes)
        dom = None
        if domain is not None:
            flat = [float(v) for pair in domain for v in pair]
            dom = (_D * len(flat))(*flat)
        self._h = _VP()
        check(lib().sgm_space_create(ctypes.byref(self._h), nd, k, n, dom,
                                     PRECISION[precision] | CHEB_METHOD[cheb]))
        self.physical_shape = self._shape(0)
        self.spectral_shape = self._shape(1)
        cheb = any(k in POLYNOMIAL for k in self.kinds)   # on any axis (the axes option of Sec. 4)
        self.real_physical = "r2c" in self.kinds or (cheb and nd == 1)
        self.real_spectral = cheb and nd == 1
        rdt = torch.float32 if precision == "f32" else torch.float64
        cdt = torch.complex64 if precision == "f32" else torch.complex128
        self.physical_dtype = rdt if self.real_physical else cdt
        self.spectral_dtype = rdt if self.real_spectral else cdt

    def _shape(self, which):
        out = (ctypes.c_int64 * len(self.kinds))()
        check(lib().sgm_space_shape(self._h, which, out))
        return tuple(int(v) for v in out)

    def solve_events(self, begin=None, end=None):
        """Record torch.cuda.Event `begin` / `end` around the elimination of every later
        physical-to-physical solve of this space (None, None clears them)."""
        def handle(ev):
            if ev is None:
                return None
            if not ev.cuda_event:   # torch creates the CUDA event on its first record
                ev.record()
            return _VP(ev.cuda_event)
        check(lib().sgm_space_solve_events(self._h, handle(begin), handle(end)))

    @property
    def cheb_method(self):
        """"tc" if axis 0 runs as the tensor-core contraction, else "fft" (Chebyshev: DCT via FFT)
        or "dense" (Legendre: the dense CUDA-core product)."""
        m = ctypes.c_int()
        check(lib().sgm_space_cheb_method(self._h, ctypes.byref(m)))
        if m.value:
            return "tc"
        return "dense" if self.kinds[0].startswith("legendre") else "fft"

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sgm_space_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers -------------------------------------------------------------------------
    def _check(self, t, shape, dtype, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        wrong = []
        if tuple(t.shape) != tuple(shape):
            wrong.append(f"shape {tuple(t.shape)} (expected {tuple(shape)})")
        if t.dtype != dtype:
            wrong.append(f"dtype {t.dtype} (expected {dtype})")
        if not t.is_contiguous():
            wrong.append(f"strides {tuple(t.stride())} (expected C-contiguous)")
        if wrong:
            raise ValueError(f"{name}: " + "; ".join(wrong))

    def empty_physical(self, device="cuda"):
        return torch.empty(self.physical_shape, dtype=self.physical_dtype, device=device)

    def empty_spectral(self, device="cuda"):
        return torch.empty(self.spectral_shape, dtype=self.spectral_dtype, device=device)

    def _run(self, fn, src, src_spec, dst_spec, out, stream, *scalars):
        self._check(src, self.spectral_shape if src_spec else self.physical_shape,
                    self.spectral_dtype if src_spec else self.physical_dtype, "input")
        if out is None:
            out = self.empty_spectral(src.device) if dst_spec else self.empty_physical(src.device)
        self._check(out, self.spectral_shape if dst_spec else self.physical_shape,
                    self.spectral_dtype if dst_spec else self.physical_dtype, "output")
        args = [self._h] + [_D(float(s)) for s in scalars] + [_ptr(src), _ptr(out), _stream(stream)]
        check(fn(*args))
        return out

    # ---- the calls of include/sgm.h ----------------------------------------------------------
    def scalar_product(self, f, out=None, stream=None):
        return self._run(lib().sgm_scalar_product, f, False, True, out, stream)

    def forward(self, u, out=None, stream=None):
        return self._run(lib().sgm_forward, u, False, True, out, stream)

    def backward(self, u_hat, out=None, stream=None):
        return self._run(lib().sgm_backward, u_hat, True, False, out, stream)

    def helmholtz_solve(self, a, b, f_tilde, out=None, stream=None):
        return self._run(lib().sgm_helmholtz_solve, f_tilde, True, True, out, stream, a, b)

    def biharmonic_solve(self, a, b, c, f_tilde, out=None, stream=None):
        return self._run(lib().sgm_biharmonic_solve, f_tilde, True, True, out, stream, a, b, c)

    def helmholtz(self, a, b, f, out=None, stream=None):
        return self._run(lib().sgm_helmholtz, f, False, False, out, stream, a, b)

    def biharmonic(self, a, b, c, f, out=None, stream=None):
        return self._run(lib().sgm_biharmonic, f, False, False, out, stream, a, b, c)

    def project_dx(self, u_hat, axis, order, out=None, stream=None):
        """project(Dx(u, axis, order), W0) (Sec. 5): the coefficients in W0 of the order-th
        derivative (0..4) along ``axis`` of the Function with coefficients u_hat.  W0 is
        ``chebyshev_space()``; the result has u_hat's shape and dtype."""
        self._check(u_hat, self.spectral_shape, self.spectral_dtype, "u_hat")
        if out is None:
            out = self.empty_spectral(u_hat.device)
        self._check(out, self.spectral_shape, self.spectral_dtype, "out")
        check(lib().sgm_project_dx(self._h, int(axis), int(order), _ptr(u_hat), _ptr(out), _stream(stream)))
        return out

    def project(self, u_hat, axis, order, target, out=None, stream=None):
        """project(Dx(u, axis, order), target) (Sec. 5) onto a target Space that differs from
        this one at most in the basis of axis 0 (regular or Shen, same family): the Galerkin
        projection's coefficients in ``target``'s spectral layout."""
        self._check(u_hat, self.spectral_shape, self.spectral_dtype, "u_hat")
        if out is None:
            out = target.empty_spectral(u_hat.device)
        target._check(out, target.spectral_shape, target.spectral_dtype, "out")
        check(lib().sgm_project(self._h, int(axis), int(order), _ptr(u_hat), target._h, _ptr(out), _stream(stream)))
        return out

    def chebyshev_space(self):
        """W0: this space with axis 0 replaced by the regular basis of its family, Chebyshev or
        Legendre (a new Space with the same sizes, domain and precision); for a Fourier-only
        space, a copy of it."""
        kinds = ["chebyshev" if k in ("dirichlet", "biharmonic", "neumann") else
                 "legendre" if k in ("legendre_dirichlet", "legendre_biharmonic") else k for k in self.kinds]
        return Space(kinds, self.sizes, domain=self.domain, precision=self.precision)


GL_SCHEMES = {"rk4": 0, "ifrk4": 1}


class GinzburgLandau:
    """Stepper for u_t = u + (1 + i beta) lap(u) - (1 + i gamma)|u|^2 u (include/sgm.h, sgm_gl_*).

    space: a square C2C x C2C Space (e.g. domain [(-50, 50), (-50, 50)]); scheme "rk4" (the
    paper's explicit RK4) or "ifrk4" (integrating-factor RK4); padding must be 1.5.
    """

    def __init__(self, space, beta, gamma, dt, scheme="rk4", padding=1.5):
        self.space = space
        self.shape = space.spectral_shape
        self.dtype = space.spectral_dtype
        self._h = _VP()
        check(lib().sgm_gl_create(ctypes.byref(self._h), space._h, float(padding), float(beta), float(gamma),
                                  float(dt), GL_SCHEMES[scheme]))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sgm_gl_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rhs(self, u_hat, out=None, stream=None):
        self.space._check(u_hat, self.shape, self.dtype, "u_hat")
        out = torch.empty_like(u_hat) if out is None else out
        self.space._check(out, self.shape, self.dtype, "out")
        check(lib().sgm_gl_rhs(self._h, _ptr(u_hat), _ptr(out), _stream(stream)))
        return out

    def step(self, u_hat, nsteps=1, stream=None):
        """Advance u_hat in place by nsteps steps."""
        self.space._check(u_hat, self.shape, self.dtype, "u_hat")
        check(lib().sgm_gl_step(self._h, _ptr(u_hat), int(nsteps), _stream(stream)))
        return u_hat


class Batch:
    """A batch of independent problems (sgm_batch_*): 1-D problems u_p'' - alpha_p u_p = f_p
    (Shen-Dirichlet, one grid per problem; f and u packed, problem p at offsets[p]:offsets[p+1])
    and optionally 2-D problems a lap(u_q) + b u_q = f_q on Shen-Dirichlet x R2C spaces (packed
    row-major N x M arrays at offsets2d[q])."""

    def __init__(self, sizes, alpha, precision="f32", autotune=True):
        self.sizes = [int(v) for v in sizes]
        self.precision = precision
        nprob = len(self.sizes)
        n = (ctypes.c_int64 * max(nprob, 1))(*self.sizes)
        a = (_D * max(nprob, 1))(*[float(v) for v in alpha])
        self._h = _VP()
        check(lib().sgm_batch_create(ctypes.byref(self._h), nprob, n, a,
                                     PRECISION[precision] | (0 if autotune else 0x40)))
        off = (ctypes.c_int64 * (nprob + 1))()
        check(lib().sgm_batch_offsets(self._h, off))
        self.offsets = [int(v) for v in off]
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        self.sizes2d = []
        self.offsets2d = [0]

    @property
    def plan(self):
        """(Bluestein prime threshold chosen by the autotuner, 0 for never; problems on that path)."""
        p, nb = ctypes.c_int(), ctypes.c_int()
        check(lib().sgm_batch_info(self._h, ctypes.byref(p), ctypes.byref(nb)))
        return p.value, nb.value

    def add_2d(self, sizes2d, a=-1.0, b=0.0):
        """Add 2-D problems of sizes [(N, M), ...] solving a lap(u) + b u = f."""
        sizes2d = [(int(N), int(M)) for N, M in sizes2d]
        flat = (ctypes.c_int64 * (2 * len(sizes2d)))(*[v for nm in sizes2d for v in nm])
        check(lib().sgm_batch_add_2d(self._h, len(sizes2d), flat, float(a), float(b)))
        self.sizes2d = sizes2d
        off = (ctypes.c_int64 * (len(sizes2d) + 1))()
        check(lib().sgm_batch_offsets_2d(self._h, off))
        self.offsets2d = [int(v) for v in off]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sgm_batch_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _packed(self, t, total, what):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.numel() == total
                and t.is_contiguous()):
            raise ValueError(f"{what} must be a contiguous CUDA {self.dtype} tensor of {total} values")
        return t

    def solve(self, f, out=None, stream=None):
        """1-D problems only, three kernel launches (sgm_batch_helmholtz)."""
        total = self.offsets[-1]
        self._packed(f, total, "f")
        out = torch.empty_like(f) if out is None else self._packed(out, total, "out")
        check(lib().sgm_batch_helmholtz(self._h, _ptr(f), _ptr(out), _stream(stream)))
        return out

    def run(self, f1=None, f2=None, out1=None, out2=None, stream=None):
        """Every problem as one CUDA graph launch (sgm_batch_run); returns (u1, u2)."""
        p1 = p2 = (None, None)
        if self.sizes:
            self._packed(f1, self.offsets[-1], "f1")
            out1 = torch.empty_like(f1) if out1 is None else self._packed(out1, self.offsets[-1], "out1")
            p1 = (_ptr(f1), _ptr(out1))
        if self.sizes2d:
            self._packed(f2, self.offsets2d[-1], "f2")
            out2 = torch.empty_like(f2) if out2 is None else self._packed(out2, self.offsets2d[-1], "out2")
            p2 = (_ptr(f2), _ptr(out2))
        check(lib().sgm_batch_run(self._h, *p1, *p2, _stream(stream)))
        return out1, out2


Batch1D = Batch


# ---- learned-closure kernels -------------------------------------------------------------------
def _vp_or_none(t):
    return _VP(t.data_ptr()) if t is not None else _VP()


CONV_RELU, CONV_OUT_F32, CONV_IN_F32 = 1, 2, 4


def conv3x3_forward(x, w, bias, y, relu, stream=None):
    """y = conv3x3(x) (+ReLU); w BF16, bias FP32, x BF16 (FP32 for a 2-channel input), y BF16 or FP32."""
    B, Cin, H, W = x.shape
    Cout = w.shape[0]
    flags = (CONV_RELU if relu else 0) | (CONV_OUT_F32 if y.dtype == torch.float32 else 0) | \
        (CONV_IN_F32 if x.dtype == torch.float32 else 0)
    check(lib().sgm_conv3x3_forward(_ptr(x), _ptr(w), _ptr(bias), _ptr(y), B, Cin, Cout, H, W, flags,
                                    _stream(stream)))
    return y


def conv3x3_backward_data(gy, w, mask, gx, stream=None):
    B, Cin, H, W = gx.shape
    Cout = w.shape[0]
    check(lib().sgm_conv3x3_backward_data(_ptr(gy), _ptr(w), _vp_or_none(mask), _ptr(gx), B, Cin, Cout, H, W,
                                          _stream(stream)))
    return gx


def conv3x3_backward_weights(gy, x, gw, gb, stream=None):
    B, Cin, H, W = x.shape
    Cout = gw.shape[0]
    flags = CONV_IN_F32 if x.dtype == torch.float32 else 0
    check(lib().sgm_conv3x3_backward_weights(_ptr(gy), _ptr(x), _ptr(gw), _ptr(gb), B, Cin, Cout, H, W, flags,
                                             _stream(stream)))


def adamw_step(w, w_bf16, g, m, v, lr, beta1, beta2, eps, weight_decay, step, stream=None):
    check(lib().sgm_adamw_step(_ptr(w), _vp_or_none(w_bf16), _ptr(g), _ptr(m), _ptr(v), w.numel(), lr, beta1, beta2,
                               eps, weight_decay, int(step), _stream(stream)))


def mse_grad(out, target, grad, loss, stream=None):
    check(lib().sgm_mse_grad(_ptr(out), _ptr(target), _ptr(grad), _ptr(loss), out.numel(), _stream(stream)))


def spectral_truncate(src, dst, stream=None):
    """src [B, Mf, Mf] complex64 -> dst [B, Mc, Mc] (wavenumbers of the coarse grid kept)."""
    B, Mf = src.shape[0], src.shape[-1]
    Mc = dst.shape[-1]
    check(lib().sgm_spectral_truncate(_ptr(src), Mf, _ptr(dst), Mc, B, _stream(stream)))
    return dst


def pack_channels(u, x, scale, stream=None):
    B, H, W = u.shape
    check(lib().sgm_pack_channels(_ptr(u), _ptr(x), B, H, W, float(scale), _stream(stream)))
    return x


AUG_TRANSPOSE, AUG_FLIP0, AUG_FLIP1 = 1, 2, 4


def augment_pack(u, d, idx, phase, sx, sy, flags, su, sd, xu, xd, stream=None):
    """Training batch of the closure: pool fields u[idx[b]], d[idx[b]] (complex64 [n, M, M]) times
    phase[b] (complex64 [B]), rolled by (sx, sy), transposed / reflected per flags (AUG_*), as FP32
    channels xu = su (Re, Im), xd = sd (Re, Im) ([B, 2, M, M]).  idx: int32 [B] on the device."""
    n, M = u.shape[0], u.shape[-1]
    B = idx.numel()
    for t, dt in ((u, torch.complex64), (d, torch.complex64), (idx, torch.int32), (phase, torch.complex64),
                  (xu, torch.float32), (xd, torch.float32)):
        if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"expected contiguous CUDA {dt}, got {t.dtype} (contiguous={t.is_contiguous()})")
    if d.shape != u.shape or phase.numel() != B or xu.shape != (B, 2, M, M) or xd.shape != (B, 2, M, M):
        raise ValueError("shapes: u, d [n, M, M]; idx, phase [B]; xu, xd [B, 2, M, M]")
    check(lib().sgm_augment_pack(_ptr(u), _ptr(d), n, M, _ptr(idx), _ptr(phase), B, int(sx), int(sy), int(flags),
                                 float(su), float(sd), _ptr(xu), _ptr(xd), _stream(stream)))


def unpack_add(d, u, scale, stream=None):
    B, H, W = u.shape
    check(lib().sgm_unpack_add(_ptr(d), _ptr(u), B, H, W, float(scale), _stream(stream)))
    return u


def tc_wait_timeouts(reset=False):
    """Bounded waits in tensor-core kernels that gave up on this device (0 when healthy)."""
    c = ctypes.c_int()
    check(lib().sgm_tc_wait_timeouts(ctypes.byref(c), 1 if reset else 0))
    return c.value


def alu_probe(precision, blocks, threads, iters, sink, stream=None):
    """Launch the FMA throughput probe (sgm_alu_probe) and return its flop count; `sink` is a
    float32/float64 CUDA tensor of at least blocks * threads elements."""
    want = torch.float64 if precision == "f64" else torch.float32
    if not sink.is_cuda or sink.dtype != want or sink.numel() < blocks * threads:
        raise ValueError(f"sink: CUDA {want} tensor of >= {blocks * threads} elements")
    fl = _D()
    check(lib().sgm_alu_probe(PRECISION[precision], blocks, threads, iters, _ptr(sink), ctypes.byref(fl),
                              _stream(stream)))
    return fl.value
