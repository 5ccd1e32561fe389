"""ctypes binding of libov (the C-ABI in include/ov.h); argument marshalling only.

Every function here has the name of the C entry point it calls. Arrays may be
numpy arrays (host memory) or CUDA torch tensors (device memory); spinors are
complex128 with shape (nrhs, 12*V) in the canonical layout 12*site + 3*spin +
colour, links complex128 with shape (V, 4, 3, 3). There is no CPU fallback:
if libov.so cannot be loaded every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libov.so")

OV_OK = 0
OV_NOT_CONVERGED = 1
OV_ERR_ARG = -1
OV_ERR_NOMEM = -2
OV_ERR_CUDA = -3
OV_ERR_BREAKDOWN = -5
OV_ERR_RH_NOCONV = -6
OV_ERR_TOO_LARGE = -7

OV_PREC_FP64 = 0
OV_PREC_FP32 = 1
OV_PREC_DF64 = 2
OV_INNER_DF64 = 0
OV_INNER_FP64 = 1
PRECISIONS = {"fp64": OV_PREC_FP64, "fp32": OV_PREC_FP32, "df64": OV_PREC_DF64}

OV_MEM_HOST = 0
OV_MEM_DEVICE = 1

OV_RECOMB_STORED = 0
OV_RECOMB_TWO_PASS = 1
OV_RECOMB_AUTO = 2


class ov_geom(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("precision", ctypes.c_int), ("t_antiperiodic", ctypes.c_int)]


class ov_opts(ctypes.Structure):
    _fields_ = [("check_interval", ctypes.c_int), ("first_check", ctypes.c_int),
                ("recombination", ctypes.c_int), ("rh_tol", ctypes.c_double), ("rh_maxit", ctypes.c_int),
                ("breakdown_tol", ctypes.c_double), ("inner_dl", ctypes.c_int), ("k_fixed", ctypes.c_int),
                ("check_schedule", ctypes.c_int), ("block_size", ctypes.c_int), ("graph_steps", ctypes.c_int),
                ("timing", ctypes.c_int), ("inner_arith", ctypes.c_int), ("relax", ctypes.c_double),
                ("overlap_checks", ctypes.c_int), ("nested", ctypes.c_int),
                ("rh_scaling", ctypes.c_int)]


class ov_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("stencil_launches", ctypes.c_longlong),
                ("update_launches", ctypes.c_longlong), ("inner_launches", ctypes.c_longlong),
                ("other_launches", ctypes.c_longlong), ("stencil_ms", ctypes.c_double),
                ("update_ms", ctypes.c_double), ("inner_ms", ctypes.c_double), ("recombine_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("outer_steps", ctypes.c_longlong),
                ("regen_steps", ctypes.c_longlong), ("checks", ctypes.c_longlong), ("block_size", ctypes.c_longlong),
                ("graph_launches", ctypes.c_longlong), ("relaxed_steps", ctypes.c_longlong),
                ("relaxed_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ov_info(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("l", ctypes.c_int), ("rh_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("err_est", ctypes.c_double), ("err_inner", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class OvError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ov_strerror(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Load libov.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libov.so not found at {LIB_PATH}: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    L.ov_default_opts.argtypes = [ctypes.POINTER(ov_opts)]
    L.ov_default_opts.restype = None
    L.ov_strerror.argtypes = [ctypes.c_int]
    L.ov_strerror.restype = ctypes.c_char_p
    L.ov_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ov_geom), vp, ctypes.c_int, ctypes.c_double,
                            ctypes.c_double, ctypes.POINTER(ov_opts), vp]
    L.ov_create.restype = ctypes.c_int
    L.ov_destroy.argtypes = [vp]
    L.ov_destroy.restype = None
    L.ov_set_opts.argtypes = [vp, ctypes.POINTER(ov_opts)]
    L.ov_set_opts.restype = ctypes.c_int
    L.ov_get_stats.argtypes = [vp, ctypes.POINTER(ov_stats)]
    L.ov_get_stats.restype = ctypes.c_int
    L.ov_reset_stats.argtypes = [vp]
    L.ov_reset_stats.restype = ctypes.c_int
    for name in ("ov_sign_apply", "ov_apply"):
        f = getattr(L, name)
        f.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                      ctypes.POINTER(ov_info)]
        f.restype = ctypes.c_int
    L.ov_deflate.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, ip]
    L.ov_deflate.restype = ctypes.c_int
    L.ov_get_deflation.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ip]
    L.ov_get_deflation.restype = ctypes.c_int
    L.ov_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                           ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, dp]
    L.ov_solve.restype = ctypes.c_int
    L.ov_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ov_geom), ctypes.POINTER(vp),
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ov_opts), vp]
    L.ov_batch_create.restype = ctypes.c_int
    L.ov_batch_sign_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(ov_info)]
    L.ov_batch_sign_apply.restype = ctypes.c_int
    L.ov_wilson_apply.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int]
    L.ov_wilson_apply.restype = ctypes.c_int
    L.ov_inner_sign.argtypes = [vp, ctypes.c_int, ctypes.c_int, ip, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, dp, ip]
    L.ov_inner_sign.restype = ctypes.c_int
    L.ov_rh_sign.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ip]
    L.ov_rh_sign.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    L.ov_mlp_forward.argtypes = [fp, ctypes.c_int, fp, fp]
    L.ov_mlp_forward.restype = ctypes.c_int
    L.ov_mlp_loss_grad.argtypes = [fp, ctypes.c_int, fp, fp, fp, fp]
    L.ov_mlp_loss_grad.restype = ctypes.c_int
    L.ov_mlp_train.argtypes = [fp, ctypes.c_int, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint, fp,
                               ctypes.c_int, fp, fp, fp]
    L.ov_mlp_train.restype = ctypes.c_int
    L.ov_set_sizer.argtypes = [vp, fp, ctypes.c_int, ctypes.c_int]
    L.ov_set_sizer.restype = ctypes.c_int
    L.ov_get_coefficients.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ip]
    L.ov_get_coefficients.restype = ctypes.c_int
    L.ov_rh_sign_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, ip, ctypes.c_double, ctypes.c_int, vp]
    L.ov_rh_sign_noalloc.restype = ctypes.c_int
    L.ov_version.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.ov_version.restype = ctypes.c_int
    _lib = L
    return L


def ov_strerror(code):
    return lib().ov_strerror(int(code)).decode()


def ov_version():
    buf = ctypes.create_string_buffer(256)
    rc = lib().ov_version(buf, 256)
    return rc, buf.value.decode()


def ov_default_opts():
    o = ov_opts()
    lib().ov_default_opts(ctypes.byref(o))
    return o


def make_opts(**kw):
    o = ov_default_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr_mem(a, writable=False):
    """(pointer, OV_MEM_*) for a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or (writable and not a.flags["WRITEABLE"]):
            raise ValueError("host arrays must be C-contiguous (and writable for outputs)")
        return ctypes.c_void_p(a.ctypes.data), OV_MEM_HOST
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if a.is_cuda:
            return ctypes.c_void_p(a.data_ptr()), OV_MEM_DEVICE
        if writable:
            raise ValueError("use numpy arrays for host outputs")
        return ctypes.c_void_p(a.data_ptr()), OV_MEM_HOST
    raise TypeError(f"unsupported array type {type(a)}")


def _check_c128(a, name):
    dt = getattr(a, "dtype", None)
    ok = dt == np.complex128
    if not ok:
        try:
            import torch
            ok = dt == torch.complex128
        except ImportError:  # pragma: no cover
            pass
    if not ok:
        raise TypeError(f"{name} must be complex128")


def ov_create(dims, links, m_w, mu, precision="fp64", t_antiperiodic=True, opts=None, stream=None):
    """Returns an opaque handle (int); links: (V,4,3,3) complex128 numpy or CUDA tensor."""
    _check_c128(links, "links")
    g = ov_geom()
    for i in range(4):
        g.dims[i] = int(dims[i])
    g.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    g.t_antiperiodic = 1 if t_antiperiodic else 0
    lp, lmem = _ptr_mem(links)
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream is not None else None
    rc = lib().ov_create(ctypes.byref(h), ctypes.byref(g), lp, lmem, float(m_w), float(mu),
                         ctypes.byref(opts) if opts is not None else None, st)
    if rc != OV_OK:
        raise OvError(rc, "ov_create")
    return h.value


def ov_destroy(h):
    if h:
        lib().ov_destroy(ctypes.c_void_p(h))


def ov_set_opts(h, opts):
    rc = lib().ov_set_opts(ctypes.c_void_p(h), ctypes.byref(opts))
    if rc != OV_OK:
        raise OvError(rc, "ov_set_opts")


def ov_get_stats(h):
    st = ov_stats()
    rc = lib().ov_get_stats(ctypes.c_void_p(h), ctypes.byref(st))
    if rc != OV_OK:
        raise OvError(rc, "ov_get_stats")
    return st.as_dict()


def ov_reset_stats(h):
    rc = lib().ov_reset_stats(ctypes.c_void_p(h))
    if rc != OV_OK:
        raise OvError(rc, "ov_reset_stats")


def _nrhs(x):
    return int(x.shape[0]) if len(x.shape) == 2 else 1


def _apply(fn, h, x, y, tol, k_max, l):
    _check_c128(x, "x")
    _check_c128(y, "y")
    nrhs = _nrhs(x)
    xp, xm = _ptr_mem(x)
    yp, ym = _ptr_mem(y, writable=True)
    if xm != ym:
        raise ValueError("x and y must both be host or both device arrays")
    infos = (ov_info * nrhs)()
    rc = fn(ctypes.c_void_p(h), nrhs, xp, yp, xm, float(tol), int(k_max), int(l), infos)
    if rc < 0:
        raise OvError(rc, fn.__name__)
    return rc, [i.as_dict() for i in infos]


def ov_sign_apply(h, x, y, tol, k_max, l):
    """y = sgn(gamma5 D_w(mu)) x; returns (status, [info per RHS])."""
    return _apply(lib().ov_sign_apply, h, x, y, tol, k_max, l)


def ov_apply(h, x, y, tol, k_max, l):
    """y = D_ov(mu) x = x + gamma5 sgn(gamma5 D_w(mu)) x."""
    return _apply(lib().ov_apply, h, x, y, tol, k_max, l)


def ov_solve(h, b, x, mass=0.0, tol=1e-8, maxit=200, sign_tol=1e-10, k_max=1000, l=120):
    """x = D(m)^{-1} b, D(m) = (1 - m/2) D_ov + m, by CG on the normal equations; every
    D and D^dag application is a nested sign apply. Returns (status, iterations, residuals)."""
    _check_c128(b, "b")
    _check_c128(x, "x")
    nrhs = _nrhs(b)
    bp, bm = _ptr_mem(b)
    xp, xm = _ptr_mem(x, writable=True)
    if bm != xm:
        raise ValueError("b and x must both be host or both device arrays")
    its = np.zeros(nrhs, dtype=np.int32)
    res = np.zeros(nrhs, dtype=np.float64)
    rc = lib().ov_solve(ctypes.c_void_p(h), nrhs, bp, xp, bm, float(mass), float(tol), int(maxit), float(sign_tol),
                        int(k_max), int(l), its.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc < 0:
        raise OvError(rc, "ov_solve")
    return rc, its, res


def ov_deflate(h, m, tol=1e-10, maxit=200, nlat=1):
    """Compute the m critical eigenpairs of every lattice and attach the converged ones
    (m = 0 detaches). Returns (status, eigenvalues (nlat, m) complex, relative residuals
    (nlat, m), pairs attached per lattice (nlat,))."""
    lam = np.zeros(2 * max(m, 1) * nlat, dtype=np.float64)
    res = np.zeros(max(m, 1) * nlat, dtype=np.float64)
    used = np.zeros(nlat, dtype=np.int32)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().ov_deflate(ctypes.c_void_p(h), int(m), float(tol), int(maxit), lam.ctypes.data_as(dp),
                          res.ctypes.data_as(dp), used.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc < 0:
        raise OvError(rc, "ov_deflate")
    lam = (lam[0::2] + 1j * lam[1::2])[:m * nlat].reshape(nlat, m)
    return rc, lam, res[:m * nlat].reshape(nlat, m), used


def ov_get_deflation(h, lattice, mcap, n):
    """(eigenvalues, R, L) of one lattice: R, L of shape (m, n) complex128 (host)."""
    lam = np.zeros(max(mcap, 1), dtype=np.complex128)
    R = np.zeros((max(mcap, 1), n), dtype=np.complex128)
    L = np.zeros((max(mcap, 1), n), dtype=np.complex128)
    m = ctypes.c_int(0)
    rc = lib().ov_get_deflation(ctypes.c_void_p(h), int(lattice), int(mcap), lam.ctypes.data, R.ctypes.data,
                                L.ctypes.data, ctypes.byref(m))
    if rc != OV_OK:
        raise OvError(rc, "ov_get_deflation")
    k = m.value
    return lam[:k], R[:k], L[:k]


def ov_wilson_apply(h, x, y, dagger=False):
    _check_c128(x, "x")
    _check_c128(y, "y")
    xp, xm = _ptr_mem(x)
    yp, ym = _ptr_mem(y, writable=True)
    if xm != ym:
        raise ValueError("x and y must both be host or both device arrays")
    rc = lib().ov_wilson_apply(ctypes.c_void_p(h), _nrhs(x), xp, yp, xm, 1 if dagger else 0)
    if rc != OV_OK:
        raise OvError(rc, "ov_wilson_apply")


def ov_inner_sign(h, k, alpha, beta, gamma, hermitian, l):
    """Inner level on tridiagonal Ritz matrices (host arrays, shape (count, ld)).

    Returns (status, c (count, ld), est_inner (count,), rh_iters (count,))."""
    alpha = np.ascontiguousarray(alpha, dtype=np.complex128)
    beta = np.ascontiguousarray(beta, dtype=np.complex128)
    gamma = np.ascontiguousarray(gamma, dtype=np.complex128)
    count, ld = alpha.shape
    kk = np.ascontiguousarray(k, dtype=np.int32)
    c = np.zeros((count, ld), dtype=np.complex128)
    est = np.zeros(count, dtype=np.float64)
    its = np.zeros(count, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().ov_inner_sign(ctypes.c_void_p(h), count, ld, kk.ctypes.data_as(ip), alpha.ctypes.data,
                             beta.ctypes.data, gamma.ctypes.data, 1 if hermitian else 0, int(l), c.ctypes.data,
                             est.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), its.ctypes.data_as(ip))
    if rc < 0 and rc != OV_ERR_RH_NOCONV:
        raise OvError(rc, "ov_inner_sign")
    return rc, c, est, its


def ov_rh_sign(h, T):
    """Roberts-Higham sign of dense matrices T (count, m, m) complex128 (host)."""
    T = np.ascontiguousarray(T, dtype=np.complex128)
    count, m, _ = T.shape
    S = np.zeros_like(T)
    its = np.zeros(count, dtype=np.int32)
    rc = lib().ov_rh_sign(ctypes.c_void_p(h), count, m, T.ctypes.data, S.ctypes.data,
                          its.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc < 0 and rc != OV_ERR_RH_NOCONV:
        raise OvError(rc, "ov_rh_sign")
    return rc, S, its


def ov_rh_sign_noalloc(T, S, rh_tol=1e-10, rh_maxit=100, stream=None):
    """Roberts-Higham sign of dense matrices without device allocation.

    T, S: CUDA complex128 tensors of shape (count, m, m) (device memory owned by the
    caller; S receives sgn(T)). For callers whose device memory is all held by their
    own pool, or that must not trigger the synchronisation an allocation can cause.
    Returns (status, iterations per matrix)."""
    tp, tm = _ptr_mem(T)
    sp, sm = _ptr_mem(S, writable=True)
    if tm != OV_MEM_DEVICE or sm != OV_MEM_DEVICE:
        raise ValueError("T and S must be CUDA tensors")
    _check_c128(T, "T")
    _check_c128(S, "S")
    # the kernel reads count * m * m entries of T and writes as many of S
    if T.dim() != 3 or T.shape[1] != T.shape[2]:
        raise ValueError(f"T must have shape (count, m, m), got {tuple(T.shape)}")
    if tuple(S.shape) != tuple(T.shape):
        raise ValueError(f"S must have T's shape {tuple(T.shape)}, got {tuple(S.shape)}")
    if S.device != T.device:
        raise ValueError("T and S must be on the same device")
    import torch

    count, m = int(T.shape[0]), int(T.shape[1])
    its = np.zeros(count, dtype=np.int32)
    with torch.cuda.device(T.device):
        # default: torch's current stream on T's device, so work queued there on T comes first
        st = stream if stream is not None else torch.cuda.current_stream(T.device).cuda_stream
        rc = lib().ov_rh_sign_noalloc(count, m, tp, sp, its.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      float(rh_tol), int(rh_maxit), ctypes.c_void_p(st) if st else None)
    if rc < 0 and rc != OV_ERR_RH_NOCONV:
        raise OvError(rc, "ov_rh_sign_noalloc")
    return rc, its


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


MLP_PARAMS = 5378


def ov_mlp_forward(theta, X):
    """Sizing network forward pass on the GPU: X (n, 16) -> (n, 2)."""
    theta = _f32(theta, (MLP_PARAMS,))
    X = _f32(X)
    Y = np.zeros((X.shape[0], 2), dtype=np.float32)
    rc = lib().ov_mlp_forward(_fp(theta), X.shape[0], _fp(X), _fp(Y))
    if rc != OV_OK:
        raise OvError(rc, "ov_mlp_forward")
    return Y


def ov_mlp_loss_grad(theta, X, Y):
    theta = _f32(theta, (MLP_PARAMS,))
    X, Y = _f32(X), _f32(Y)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_PARAMS, dtype=np.float32)
    rc = lib().ov_mlp_loss_grad(_fp(theta), X.shape[0], _fp(X), _fp(Y), _fp(loss), _fp(grad))
    if rc != OV_OK:
        raise OvError(rc, "ov_mlp_loss_grad")
    return float(loss[0]), grad


def ov_mlp_train(theta, X, Y, epochs, batch=0, lr=1e-3, seed=1, Xv=None, Yv=None):
    """Train on the GPU (Adam); returns (theta, training loss per epoch) or, with validation
    data, (theta of the best validation epoch, training losses, validation losses)."""
    th = _f32(theta, (MLP_PARAMS,)).copy()
    X, Y = _f32(X), _f32(Y)
    hist = np.zeros(epochs, dtype=np.float32)
    if Xv is None:
        rc = lib().ov_mlp_train(_fp(th), X.shape[0], _fp(X), _fp(Y), int(epochs), int(batch), float(lr), int(seed),
                                _fp(hist), 0, None, None, None)
        if rc != OV_OK:
            raise OvError(rc, "ov_mlp_train")
        return th, hist
    Xv, Yv = _f32(Xv), _f32(Yv)
    vh = np.zeros(epochs, dtype=np.float32)
    rc = lib().ov_mlp_train(_fp(th), X.shape[0], _fp(X), _fp(Y), int(epochs), int(batch), float(lr), int(seed),
                            _fp(hist), Xv.shape[0], _fp(Xv), _fp(Yv), _fp(vh))
    if rc != OV_OK:
        raise OvError(rc, "ov_mlp_train")
    return th, hist, vh


def ov_set_sizer(h, theta, l_min=8, l_max=120):
    if theta is None:
        rc = lib().ov_set_sizer(ctypes.c_void_p(h), None, int(l_min), int(l_max))
    else:
        th = _f32(theta, (MLP_PARAMS,))
        rc = lib().ov_set_sizer(ctypes.c_void_p(h), _fp(th), int(l_min), int(l_max))
    if rc != OV_OK:
        raise OvError(rc, "ov_set_sizer")


def ov_get_coefficients(h, rhs, kcap):
    """(alpha, beta, gamma) of the last apply for one RHS, index 0 = step 1."""
    a = np.zeros(kcap, dtype=np.complex128)
    b = np.zeros(kcap, dtype=np.complex128)
    g = np.zeros(kcap, dtype=np.complex128)
    k = ctypes.c_int(0)
    rc = lib().ov_get_coefficients(ctypes.c_void_p(h), int(rhs), int(kcap), a.ctypes.data, b.ctypes.data,
                                   g.ctypes.data, ctypes.byref(k))
    if rc != OV_OK:
        raise OvError(rc, "ov_get_coefficients")
    return a[:k.value], b[:k.value], g[:k.value]


def ov_batch_create(dims_list, links_list, m_w_list, mu_list, precision="fp32", t_antiperiodic=True, opts=None,
                    stream=None):
    """Handle for a batch of independent lattices (one source each)."""
    n = len(dims_list)
    geoms = (ov_geom * n)()
    keep = []
    ptrs = (ctypes.c_void_p * n)()
    mem = None
    for i in range(n):
        for d in range(4):
            geoms[i].dims[d] = int(dims_list[i][d])
        geoms[i].precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        geoms[i].t_antiperiodic = 1 if t_antiperiodic else 0
        _check_c128(links_list[i], "links")
        p, m = _ptr_mem(links_list[i])
        if mem is None:
            mem = m
        elif m != mem:
            raise ValueError("links must all be host or all device arrays")
        ptrs[i] = p.value
        keep.append(links_list[i])
    mw = (ctypes.c_double * n)(*[float(v) for v in m_w_list])
    mu = (ctypes.c_double * n)(*[float(v) for v in mu_list])
    h = ctypes.c_void_p()
    rc = lib().ov_batch_create(ctypes.byref(h), n, geoms, ptrs, mem, mw, mu,
                               ctypes.byref(opts) if opts is not None else None,
                               ctypes.c_void_p(stream) if stream is not None else None)
    if rc != OV_OK:
        raise OvError(rc, "ov_batch_create")
    return h.value


def ov_batch_sign_apply(h, xs, ys, tol, k_max, l):
    """xs, ys: lists of complex128 arrays (all host numpy or all CUDA tensors)."""
    n = len(xs)
    xp = (ctypes.c_void_p * n)()
    yp = (ctypes.c_void_p * n)()
    mem = None
    for i in range(n):
        _check_c128(xs[i], "x")
        _check_c128(ys[i], "y")
        p, m = _ptr_mem(xs[i])
        q, m2 = _ptr_mem(ys[i], writable=True)
        if m != m2 or (mem is not None and m != mem):
            raise ValueError("x and y must all be host or all device arrays")
        mem = m
        xp[i] = p.value
        yp[i] = q.value
    infos = (ov_info * n)()
    rc = lib().ov_batch_sign_apply(ctypes.c_void_p(h), xp, yp, mem, float(tol), int(k_max), int(l), infos)
    if rc < 0:
        raise OvError(rc, "ov_batch_sign_apply")
    return rc, [i.as_dict() for i in infos]


class Overlap:
    """Owner of one handle: y = sgn(gamma5 D_w(mu)) x and D_ov(mu) x for one gauge field."""

    def __init__(self, dims, links, m_w, mu, precision="fp64", t_antiperiodic=True, opts=None, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.h = ov_create(self.dims, links, m_w, mu, precision, t_antiperiodic, opts, stream)

    def close(self):
        if self.h:
            ov_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **kw):
        ov_set_opts(self.h, make_opts(**kw))

    def stats(self):
        return ov_get_stats(self.h)

    def set_sizer(self, theta, l_min=8, l_max=120):
        ov_set_sizer(self.h, theta, l_min, l_max)

    def coefficients(self, rhs, kcap):
        return ov_get_coefficients(self.h, rhs, kcap)

    def reset_stats(self):
        ov_reset_stats(self.h)

    def sign_apply(self, x, y, tol, k_max, l):
        return ov_sign_apply(self.h, x, y, tol, k_max, l)

    def apply(self, x, y, tol, k_max, l):
        return ov_apply(self.h, x, y, tol, k_max, l)

    def deflate(self, m, tol=1e-10, maxit=200):
        rc, lam, res, used = ov_deflate(self.h, m, tol, maxit)
        return rc, lam[0], res[0]

    def deflation(self, mcap=64):
        n = 12 * int(np.prod(self.dims))
        return ov_get_deflation(self.h, 0, mcap, n)

    def solve(self, b, x, mass=0.0, tol=1e-8, maxit=200, sign_tol=1e-10, k_max=1000, l=120):
        return ov_solve(self.h, b, x, mass, tol, maxit, sign_tol, k_max, l)

    def wilson_apply(self, x, y, dagger=False):
        return ov_wilson_apply(self.h, x, y, dagger)
