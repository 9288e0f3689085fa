"""Python binding of libse2ot.so (include/se2ot.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Tensors are torch tensors whose
storage the library reads or writes through raw pointers; PyTorch supplies device memory and
the current CUDA stream, nothing else.  If the library is missing the import fails: there is
no fallback implementation.

Layout of every field: [batch, ny, nx, ntheta], C-contiguous (orientation innermost).
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libse2ot.so")

SE2OT_OK = 0
SE2OT_EINVAL = 1
SE2OT_ENOMEM = 2
SE2OT_ECUDA = 3
SE2OT_ENONFINITE = 4
SE2OT_ENOTCONV = 5
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ENOTCONV",
                6: "ETIMEOUT", 7: "EBUSY", 8: "ESHUTDOWN"}
SE2OT_FP32 = 0
SE2OT_BF16TC = 1
SE2OT_BOUNDARY_ZERO = 0
SE2OT_BOUNDARY_PERIODIC = 1
SE2OT_DIST_RHO_B, SE2OT_DIST_RHO_C = 0, 1
SE2OT_FLAG_TIME_CONV = 1
SE2OT_FLAG_BATCH_ONE_LAUNCH = 2
SE2OT_FLAG_BATCH_PER_RADIUS = 4


class se2ot_kernel_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("radius", ctypes.c_int), ("w1", ctypes.c_double), ("w2", ctypes.c_double),
                ("w3", ctypes.c_double), ("eps", ctypes.c_double), ("boundary", ctypes.c_int),
                ("distance", ctypes.c_int)]


class se2ot_solve_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("tol_viol", ctypes.c_double), ("precision", ctypes.c_int), ("flags", ctypes.c_int),
                ("refine_iters", ctypes.c_int)]


class se2ot_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("mass", ctypes.c_double), ("viol", ctypes.c_double),
                ("ms", ctypes.c_double), ("voxel_iters_per_s", ctypes.c_double),
                ("conv_ms", ctypes.c_double), ("conv_launches", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("redo_outputs", ctypes.c_longlong),
                ("evaluated_terms", ctypes.c_longlong), ("logscale_min", ctypes.c_double),
                ("logscale_max", ctypes.c_double), ("tc_tiles", ctypes.c_longlong),
                ("tc_fallback_tiles", ctypes.c_longlong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class se2ot_w2_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cost", ctypes.c_double), ("dual", ctypes.c_double),
                ("mass", ctypes.c_double), ("viol", ctypes.c_double), ("ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("redo_outputs", ctypes.c_longlong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SE2OTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_LIB = None


def lib():
    """Load libse2ot.so (built in-tree by paper_2402_15322_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError("libse2ot.so not found at %s; build it with "
                          "`python -m paper_2402_15322_gb300.build`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.se2ot_kernel_build.argtypes = [ctypes.POINTER(se2ot_kernel_desc), vp, ctypes.POINTER(vp)]
    L.se2ot_kernel_destroy.argtypes = [vp]
    L.se2ot_kernel_taps.argtypes = [vp, vp]
    L.se2ot_apply.argtypes = [vp, vp, vp, i, i, vp]
    L.se2ot_apply_log.argtypes = [vp, vp, vp, i, i, vp]
    L.se2ot_barycenter.argtypes = [vp, i, vp, vp, ctypes.POINTER(se2ot_solve_opts), vp,
                                   ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_interpolate.argtypes = [vp, vp, vp, d, ctypes.POINTER(se2ot_solve_opts), vp,
                                    ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_state_export.argtypes = [vp, i, vp, vp, vp, vp]
    L.se2ot_w2.argtypes = [vp, vp, vp, ctypes.POINTER(se2ot_solve_opts), ctypes.POINTER(se2ot_w2_result), vp]
    L.se2ot_project.argtypes = [vp, vp, i, i, i, i, vp]
    L.se2ot_jko.argtypes = [vp, vp, d, d, i, ctypes.POINTER(se2ot_solve_opts), vp, ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_lift_field.argtypes = [vp, vp, i, i, i, vp]
    L.se2ot_reconstruct_field.argtypes = [vp, vp, i, i, i, vp]
    L.se2ot_interpolate_signed.argtypes = [vp, vp, vp, d, ctypes.POINTER(se2ot_solve_opts), vp,
                                           ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_interpolate_batched.argtypes = [i, ctypes.POINTER(se2ot_kernel_desc), ctypes.POINTER(vp),
                                            ctypes.POINTER(vp), ctypes.POINTER(d),
                                            ctypes.POINTER(se2ot_solve_opts), ctypes.POINTER(vp),
                                            ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_barycenter_noalloc.argtypes = [ctypes.POINTER(se2ot_kernel_desc), i, vp, vp,
                                           ctypes.POINTER(se2ot_solve_opts), vp,
                                           ctypes.POINTER(se2ot_stats), vp]
    L.se2ot_serve_create.argtypes = [ctypes.c_size_t, i, i, ctypes.POINTER(vp)]
    L.se2ot_serve_submit.argtypes = [vp, ctypes.POINTER(se2ot_kernel_desc), i, vp, ctypes.POINTER(d),
                                     ctypes.POINTER(se2ot_solve_opts), ctypes.POINTER(ctypes.c_uint64)]
    L.se2ot_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i)]
    L.se2ot_serve_wait.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(se2ot_stats), i]
    L.se2ot_serve_destroy.argtypes = [vp]
    L.se2ot_sfu_ex2_rate.argtypes = [ctypes.POINTER(d), vp]
    L.se2ot_batch_tuning.argtypes = [ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(d)]
    L.se2ot_last_error.restype = ctypes.c_char_p
    L.se2ot_version.restype = ctypes.c_char_p
    for name in ("se2ot_kernel_build", "se2ot_kernel_destroy", "se2ot_kernel_taps", "se2ot_apply",
                 "se2ot_apply_log", "se2ot_barycenter", "se2ot_interpolate", "se2ot_barycenter_noalloc",
                 "se2ot_state_export", "se2ot_interpolate_batched", "se2ot_serve_create", "se2ot_serve_submit",
                 "se2ot_serve_poll", "se2ot_serve_wait", "se2ot_serve_destroy", "se2ot_sfu_ex2_rate",
                 "se2ot_batch_tuning"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _check(status):
    if status != SE2OT_OK:
        raise SE2OTError(status, se2ot_last_error())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype):
    if t.dtype != dtype:
        raise TypeError("expected %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _shape(desc):
    return (desc.ny, desc.nx, desc.ntheta)


def _need(t, shape, what, cuda=None, device=None):
    """Argument check before a raw pointer is handed to the library: the C side reads and writes
    exactly prod(shape) elements, so a smaller tensor would be an out-of-bounds access."""
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (what, tuple(t.shape), tuple(shape)))
    if cuda is True and not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if device is not None and t.is_cuda and t.device != device:
        raise ValueError("%s is on %s, expected %s" % (what, t.device, device))


def _weights(lam, n):
    lam = [float(x) for x in lam]
    if len(lam) != n:
        raise ValueError("%d weights for %d measures" % (len(lam), n))
    return (ctypes.c_double * n)(*lam)


def se2ot_sfu_ex2_rate(stream=None):
    """Measured ex2 results per second of the current device (the SFU ceiling of the log-domain
    convolution's evaluated terms)."""
    v = ctypes.c_double()
    _check(lib().se2ot_sfu_ex2_rate(ctypes.byref(v), _stream(stream)))
    return v.value


def se2ot_last_error():
    return lib().se2ot_last_error().decode()


def se2ot_version():
    return lib().se2ot_version().decode()


class Kernel:
    """Owner of an se2ot_kernel handle (tap tables and workspace on the current device)."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc

    @property
    def shape(self):
        d = self.desc
        return (d.ny, d.nx, d.ntheta)

    @property
    def V(self):
        d = self.desc
        return d.nx * d.ny * d.ntheta

    def close(self):
        if self.handle:
            lib().se2ot_kernel_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(nx, ny, ntheta, radius, w=(1.0, 3.0, 0.5), eps=1e-3, periodic=False, distance="rho_b"):
    """Kernel descriptor; distance "rho_b" (half-angle, the paper's) or "rho_c" (logarithmic)."""
    if distance not in ("rho_b", "rho_c"):
        raise ValueError("distance must be 'rho_b' or 'rho_c'")
    return se2ot_kernel_desc(int(nx), int(ny), int(ntheta), int(radius), float(w[0]), float(w[1]),
                             float(w[2]), float(eps),
                             SE2OT_BOUNDARY_PERIODIC if periodic else SE2OT_BOUNDARY_ZERO,
                             SE2OT_DIST_RHO_C if distance == "rho_c" else SE2OT_DIST_RHO_B)


def se2ot_kernel_build(desc, stream=None):
    h = ctypes.c_void_p()
    _check(lib().se2ot_kernel_build(ctypes.byref(desc), _stream(stream), ctypes.byref(h)))
    return Kernel(h, desc)


def se2ot_kernel_destroy(kernel):
    kernel.close()


def se2ot_kernel_taps(kernel):
    """Tap table as a float32 CPU tensor [o, i, dy + r, dx + r] of log2 K."""
    d = kernel.desc
    D = 2 * d.radius + 1
    out = torch.empty((d.ntheta, d.ntheta, D, D), dtype=torch.float32)
    _check(lib().se2ot_kernel_taps(kernel.handle, ctypes.c_void_p(out.data_ptr())))
    return out


def se2ot_apply(kernel, f, out=None, stream=None, precision=SE2OT_FP32):
    """out = K * f for f of shape [batch, ny, nx, ntheta] (float32, CUDA); precision SE2OT_FP32 or
    SE2OT_BF16TC (tensor cores)."""
    batch = f.numel() // kernel.V
    _need(f, (batch,) + kernel.shape, "f", cuda=True)
    if out is None:
        out = torch.empty_like(f)
    _need(out, tuple(f.shape), "out", cuda=True, device=f.device)
    _check(lib().se2ot_apply(kernel.handle, _ptr(f, torch.float32), _ptr(out, torch.float32), batch,
                             int(precision), _stream(stream)))
    return out


def se2ot_apply_log(kernel, lf, out=None, stream=None, precision=SE2OT_FP32):
    """out = log(K * exp(lf)) (float64, CUDA); precision as in se2ot_apply."""
    batch = lf.numel() // kernel.V
    _need(lf, (batch,) + kernel.shape, "lf", cuda=True)
    if out is None:
        out = torch.empty_like(lf)
    _need(out, tuple(lf.shape), "out", cuda=True, device=lf.device)
    _check(lib().se2ot_apply_log(kernel.handle, _ptr(lf, torch.float64), _ptr(out, torch.float64), batch,
                                 int(precision), _stream(stream)))
    return out


def solve_opts(max_iters=100, check_every=0, tol_viol=0.0, precision=SE2OT_FP32, flags=0, refine_iters=0):
    return se2ot_solve_opts(int(max_iters), int(check_every), float(tol_viol), int(precision), int(flags),
                            int(refine_iters))


def se2ot_barycenter(kernel, mu, lam, opts=None, out=None, stream=None, raise_on_error=True):
    """Barycenter of mu [n, ny, nx, ntheta] (float32, CUDA or pinned/pageable CPU) with weights
    lam (n floats).  Returns (bary, stats dict, status)."""
    n = mu.shape[0]
    _need(mu, (n,) + kernel.shape, "mu")
    if out is None:
        out = torch.empty(mu.shape[1:], dtype=torch.float32, device=mu.device)
    _need(out, kernel.shape, "out")
    lam_c = _weights(lam, n)
    st = se2ot_stats()
    status = lib().se2ot_barycenter(kernel.handle, n, _ptr(mu, torch.float32), lam_c,
                                    ctypes.byref(opts if opts is not None else solve_opts()),
                                    _ptr(out, torch.float32), ctypes.byref(st), _stream(stream))
    if raise_on_error:
        _check(status)
    return out, st.as_dict(), status


def se2ot_state_export(kernel, n, device="cuda", stream=None):
    """Natural logs of v_i, d_i ([n, ny, nx, ntheta]) and mu ([ny, nx, ntheta]) after the last solve,
    as float64 CUDA tensors."""
    shape = kernel.shape
    lv = torch.empty((n,) + shape, dtype=torch.float64, device=device)
    ld = torch.empty_like(lv)
    lmu = torch.empty(shape, dtype=torch.float64, device=device)
    _check(lib().se2ot_state_export(kernel.handle, int(n), _ptr(lv, torch.float64), _ptr(ld, torch.float64),
                                    _ptr(lmu, torch.float64), _stream(stream)))
    return lv, ld, lmu


def se2ot_w2(kernel, mu, nu, opts=None, stream=None, raise_on_error=True):
    """Entropic transport between mu and nu (Sec. 4.1): returns (result dict with cost <c, pi>,
    dual, plan mass, first-marginal violation, iterations; status)."""
    _need(mu, kernel.shape, "mu")
    _need(nu, kernel.shape, "nu")
    res = se2ot_w2_result()
    status = lib().se2ot_w2(kernel.handle, _ptr(mu, torch.float32), _ptr(nu, torch.float32),
                            ctypes.byref(opts if opts is not None else solve_opts()), ctypes.byref(res),
                            _stream(stream))
    if raise_on_error:
        _check(status)
    return res.as_dict(), status


def se2ot_jko(kernel, mu0, tau, m, steps, opts=None, out=None, stream=None, raise_on_error=True):
    """`steps` entropic JKO steps of the porous-medium energy sum mu^m / (m - 1) from mu0 [ny, nx, nt]
    (opts.max_iters scaling iterations per step).  Returns (mu, stats dict, status)."""
    _need(mu0, kernel.shape, "mu0")
    if out is None:
        out = torch.empty_like(mu0)
    _need(out, kernel.shape, "out")
    st = se2ot_stats()
    status = lib().se2ot_jko(kernel.handle, _ptr(mu0, torch.float32), float(tau), float(m), int(steps),
                             ctypes.byref(opts if opts is not None else solve_opts()), _ptr(out, torch.float32),
                             ctypes.byref(st), _stream(stream))
    if raise_on_error:
        _check(status)
    return out, st.as_dict(), status


def se2ot_project(U, stream=None):
    """P(U) = sum over the orientation bins: U [..., ny, nx, nt] (CUDA float32) -> [..., ny, nx]."""
    ny, nx, nt = U.shape[-3:]
    batch = U.numel() // (ny * nx * nt)
    P = torch.empty(U.shape[:-1], dtype=torch.float32, device=U.device)
    _check(lib().se2ot_project(_ptr(U, torch.float32), _ptr(P, torch.float32), batch, nx, ny, nt, _stream(stream)))
    return P


def se2ot_lift_field(v, ntheta, stream=None):
    """Orientation-field lift: v [ny, nx, 2] (CUDA float32) -> U [ny, nx, ntheta]."""
    ny, nx = v.shape[:2]
    U = torch.empty((ny, nx, ntheta), dtype=torch.float32, device=v.device)
    _check(lib().se2ot_lift_field(_ptr(v, torch.float32), _ptr(U, torch.float32), nx, ny, ntheta, _stream(stream)))
    return U


def se2ot_reconstruct_field(U, stream=None):
    """Field reconstruction: U [ny, nx, nt] (CUDA float32) -> v [ny, nx, 2]."""
    ny, nx, nt = U.shape
    v = torch.empty((ny, nx, 2), dtype=torch.float32, device=U.device)
    _check(lib().se2ot_reconstruct_field(_ptr(U, torch.float32), _ptr(v, torch.float32), nx, ny, nt, _stream(stream)))
    return v


def se2ot_interpolate_signed(kernel, U0, U1, t, opts=None, stream=None, raise_on_error=True):
    """Signed-score interpolation b_t = m+_t P(Phi_t(U0+, U1+)) - m-_t P(Phi_t(U0-, U1-)).
    Returns (b [ny, nx], [stats of the positive part, of the negative part], status)."""
    _need(U0, kernel.shape, "U0", cuda=True)
    _need(U1, kernel.shape, "U1", cuda=True, device=U0.device)
    ny, nx = U0.shape[:2]
    b = torch.empty((ny, nx), dtype=torch.float32, device=U0.device)
    st = (se2ot_stats * 2)()
    status = lib().se2ot_interpolate_signed(kernel.handle, _ptr(U0, torch.float32), _ptr(U1, torch.float32), float(t),
                                            ctypes.byref(opts if opts is not None else solve_opts()), _ptr(b, torch.float32),
                                            st, _stream(stream))
    if raise_on_error:
        _check(status)
    return b, [st[0].as_dict(), st[1].as_dict()], status


def se2ot_interpolate(kernel, mu0, mu1, t, opts=None, out=None, stream=None, raise_on_error=True):
    """Phi_t(mu0, mu1): the barycenter with weights (1 - t, t)."""
    _need(mu0, kernel.shape, "mu0")
    _need(mu1, kernel.shape, "mu1")
    if out is None:
        out = torch.empty_like(mu0)
    _need(out, kernel.shape, "out")
    st = se2ot_stats()
    status = lib().se2ot_interpolate(kernel.handle, _ptr(mu0, torch.float32), _ptr(mu1, torch.float32),
                                     float(t), ctypes.byref(opts if opts is not None else solve_opts()),
                                     _ptr(out, torch.float32), ctypes.byref(st), _stream(stream))
    if raise_on_error:
        _check(status)
    return out, st.as_dict(), status


NOALLOC_SCRATCH_BYTES = 16 << 20


def se2ot_barycenter_noalloc(desc, mu, lam, opts=None, out=None, stream=None, raise_on_error=True):
    """Barycenter without any device allocation by the library (for callers that cannot
    allocate): mu [n, ny, nx, ntheta] and out must be CUDA tensors; the tap table and the
    workspace live in the library's static 16 MiB device array, shared by every call.
    Returns (bary, stats dict, status)."""
    n = mu.shape[0]
    _need(mu, (n,) + _shape(desc), "mu", cuda=True)
    if out is None:
        out = torch.empty(mu.shape[1:], dtype=torch.float32, device=mu.device)
    _need(out, _shape(desc), "out", cuda=True, device=mu.device)
    lam_c = _weights(lam, n)
    st = se2ot_stats()
    status = lib().se2ot_barycenter_noalloc(ctypes.byref(desc), n, _ptr(mu, torch.float32), lam_c,
                                            ctypes.byref(opts if opts is not None else solve_opts()),
                                            _ptr(out, torch.float32), ctypes.byref(st), _stream(stream))
    if raise_on_error:
        _check(status)
    return out, st.as_dict(), status


def se2ot_interpolate_batched(descs, mu0s, mu1s, ts, opts=None, outs=None, stream=None, raise_on_error=True):
    """Batched interpolations: descs, mu0s, mu1s (CUDA float32 tensors [ny, nx, ntheta] per problem),
    ts (floats).  Returns (outs, list of stats dicts, status)."""
    n = len(descs)
    if not (len(mu0s) == len(mu1s) == len(ts) == n):
        raise ValueError("descs, mu0s, mu1s and ts must have the same length")
    for p in range(n):
        _need(mu0s[p], _shape(descs[p]), "mu0s[%d]" % p, cuda=True)
        _need(mu1s[p], _shape(descs[p]), "mu1s[%d]" % p, cuda=True, device=mu0s[p].device)
    if outs is None:
        outs = [torch.empty_like(m) for m in mu0s]
    for p in range(n):
        _need(outs[p], _shape(descs[p]), "outs[%d]" % p, cuda=True, device=mu0s[p].device)
    darr = (se2ot_kernel_desc * n)(*descs)
    p0 = (ctypes.c_void_p * n)(*[_ptr(m, torch.float32).value for m in mu0s])
    p1 = (ctypes.c_void_p * n)(*[_ptr(m, torch.float32).value for m in mu1s])
    po = (ctypes.c_void_p * n)(*[_ptr(m, torch.float32).value for m in outs])
    tt = (ctypes.c_double * n)(*[float(x) for x in ts])
    st = (se2ot_stats * n)()
    status = lib().se2ot_interpolate_batched(n, darr, p0, p1, tt,
                                             ctypes.byref(opts if opts is not None else solve_opts()),
                                             po, st, _stream(stream))
    if raise_on_error:
        _check(status)
    return outs, [s.as_dict() for s in st], status


def se2ot_batch_tuning():
    """(form, ms per iteration per radius, ms per iteration in one launch) of the last tuned batch;
    form 1 = per radius, 2 = one launch, 0 = none tuned."""
    f, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(lib().se2ot_batch_tuning(ctypes.byref(f), ctypes.byref(a), ctypes.byref(b)))
    return f.value, a.value, b.value


SE2OT_ETIMEOUT = 6
SE2OT_ESHUTDOWN = 8


class Server:
    """se2ot_serve_*: continuous-batching request loop for barycenter solves."""

    def __init__(self, budget_bytes, max_slots=8, device=0):
        h = ctypes.c_void_p()
        _check(lib().se2ot_serve_create(int(budget_bytes), int(max_slots), int(device), ctypes.byref(h)))
        self.handle = h
        self._shapes = {}   # ticket -> result shape, to check the tensor wait() writes into

    def submit(self, desc, mu, lam, opts=None):
        """Queue a barycenter of mu [n, ny, nx, ntheta] (float32, CPU or CUDA); returns a ticket."""
        n = mu.shape[0]
        _need(mu, (n,) + _shape(desc), "mu")
        t = ctypes.c_uint64()
        lam_c = _weights(lam, n)
        _check(lib().se2ot_serve_submit(self.handle, ctypes.byref(desc), n, _ptr(mu, torch.float32), lam_c,
                                        ctypes.byref(opts if opts is not None else solve_opts()), ctypes.byref(t)))
        self._shapes[t.value] = _shape(desc)
        return t.value

    def poll(self, ticket):
        d = ctypes.c_int()
        _check(lib().se2ot_serve_poll(self.handle, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, out, timeout_ms=-1):
        """Copy the result into out (float32 tensor, CPU or CUDA); returns (stats dict, status)."""
        if out is not None and ticket in self._shapes:
            _need(out, self._shapes[ticket], "out")
        st = se2ot_stats()
        status = lib().se2ot_serve_wait(self.handle, ticket, _ptr(out, torch.float32) if out is not None else None,
                                        ctypes.byref(st), int(timeout_ms))
        if status != SE2OT_ETIMEOUT:
            self._shapes.pop(ticket, None)
        return st.as_dict(), status

    def close(self):
        if self.handle:
            lib().se2ot_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
