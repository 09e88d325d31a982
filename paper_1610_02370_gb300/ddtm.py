"""Thin ctypes binding of libddtm (include/ddtm.h): same entry-point names,
argument marshalling only.  Every computation runs in the CUDA library.

Importing this module loads ``libddtm.so`` and raises ImportError if it has not
been built (``python -m paper_1610_02370_gb300.build``); there is no fallback.

Arrays: numpy arrays (host) or torch tensors (host or CUDA), complex128 and
C-contiguous, in the canonical layouts of the header.  A CUDA tensor is passed
as a device pointer (DDTM_LOC_DEVICE), anything else as host memory.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddtm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libddtm.so is not built: run python -m paper_1610_02370_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOCONV, ERR_NAN, ERR_STATE, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
LOC_HOST, LOC_DEVICE = 0, 1
PREC_F64, PREC_F32, PREC_F16 = 0, 1, 2
MAX_LEVELS = 4
ERROR_NAMES = {ERR_ARG: "ERR_ARG", ERR_CUDA: "ERR_CUDA", ERR_OOM: "ERR_OOM", ERR_NOCONV: "ERR_NOCONV",
               ERR_NAN: "ERR_NAN", ERR_STATE: "ERR_STATE", ERR_TIMEOUT: "ERR_TIMEOUT"}


class ddtm_params(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("n_setup", ctypes.c_int), ("nv", ctypes.c_int * MAX_LEVELS),
                ("block", (ctypes.c_int * 4) * MAX_LEVELS), ("post_smooth", ctypes.c_int), ("nmr", ctypes.c_int),
                ("kcycle_restart", ctypes.c_int), ("kcycle_max_restarts", ctypes.c_int),
                ("kcycle_tol", ctypes.c_double), ("coarse_restart", ctypes.c_int),
                ("coarse_max_restarts", ctypes.c_int), ("coarse_tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("outer_restart", ctypes.c_int), ("outer_max_iters", ctypes.c_int), ("outer_tol", ctypes.c_double),
                ("restart_tol", ctypes.c_double), ("smoother_prec", ctypes.c_int), ("coarse_prec", ctypes.c_int)]


class ddtm_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("coarse_iters", ctypes.c_long),
                ("max_relres", ctypes.c_double), ("solve_s", ctypes.c_double), ("setup_s", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "ddtm_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I), _I]),
    "ddtm_destroy": (_I, [_P]),
    "ddtm_last_error": (ctypes.c_char_p, [_P]),
    "ddtm_set_stream": (_I, [_P, _P]),
    "ddtm_default_params": (_I, [ctypes.POINTER(ddtm_params)]),
    "ddtm_get_params": (_I, [_P, ctypes.POINTER(ddtm_params)]),
    "ddtm_set_params": (_I, [_P, ctypes.POINTER(ddtm_params)]),
    "ddtm_load_gauge": (_I, [_P, _P, _I, _D, _D]),
    "ddtm_apply_D": (_I, [_P, _P, _P, _I, _D, _I, _I]),
    "ddtm_set_boundary_phases": (_I, [_P, ctypes.POINTER(_D)]),
    "ddtm_apply_D_noalloc": (_I, [_P, _P, _P, _D, _I]),
    "ddtm_sap": (_I, [_P, _P, _P, _I, _D, _I, _I, _I, _I]),
    "ddtm_field_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "ddtm_field_destroy": (_I, [_P]),
    "ddtm_field_import": (_I, [_P, _P, _P, _I]),
    "ddtm_field_export": (_I, [_P, _P, _P, _I]),
    "ddtm_apply_D_field": (_I, [_P, _P, _P, _D]),
    "ddtm_sap_field": (_I, [_P, _P, _P, _D, _I, _I]),
    "ddtm_setup": (_I, [_P, _D, ctypes.c_uint64]),
    "ddtm_setup_update": (_I, [_P, _D, _I]),
    "ddtm_set_test_vectors": (_I, [_P, _I, _P, _I, _I]),
    "ddtm_build_coarse": (_I, [_P]),
    "ddtm_get_prolongator": (_I, [_P, _I, _P, _I]),
    "ddtm_restrict": (_I, [_P, _I, _P, _P, _I, _I]),
    "ddtm_prolong": (_I, [_P, _I, _P, _P, _I, _I]),
    "ddtm_apply_Dc": (_I, [_P, _I, _P, _P, _I, _D, _I]),
    "ddtm_coarse_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I)]),
    "ddtm_coarse_solve_batch": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(_I)]),
    "ddtm_sap_coarse": (_I, [_P, _I, _P, _P, _I, _D, _I, _I, _I]),
    "ddtm_solve": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(ddtm_solve_info)]),
    "ddtm_eo_cg": (_I, [_P, _P, _P, _I, _D, _D, _I, _I, ctypes.POINTER(ddtm_solve_info)]),
    "ddtm_save_setup": (_I, [_P, ctypes.c_char_p]),
    "ddtm_load_setup": (_I, [_P, ctypes.c_char_p]),
    "ddtm_timer_enable": (_I, [_P, _I]),
    "ddtm_timer_reset": (_I, [_P]),
    "ddtm_timer_report": (_I, [_P, ctypes.c_char_p, _I]),
    "ddtm_measure_fma_peak": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "ddtm_set_memory_limit": (_I, [ctypes.c_size_t]),
    "ddtm_release_workspace": (_I, [_P]),
    "ddtm_set_option": (_I, [_P, ctypes.c_char_p, _I]),
    "ddtm_get_option": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_I)]),
    "ddtm_autotune_report": (_I, [ctypes.c_char_p, _I]),
    "ddtm_memory_in_use": (_I, [ctypes.POINTER(ctypes.c_size_t)]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class DDTMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, code), msg))
        self.code = code


def _check(ctx, code):
    if code != OK:
        msg = _lib.ddtm_last_error(ctx).decode() if ctx else ""
        raise DDTMError(code, msg)


def _buf(a, writable=False):
    """(pointer, loc) of a complex128 C-contiguous numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.complex128 or not a.is_contiguous():
                raise TypeError("expected a contiguous complex128 tensor")
            return a.data_ptr(), (LOC_DEVICE if a.is_cuda else LOC_HOST)
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous complex128 numpy array or torch tensor")
    if writable and not a.flags.writeable:
        raise TypeError("output array is read-only")
    return a.ctypes.data, LOC_HOST


def _same_loc(*bufs):
    locs = {b[1] for b in bufs}
    if len(locs) != 1:
        raise TypeError("all arrays of one call must live on the same side (host or device)")
    return locs.pop()


# ---- entry points (same names as the C ABI) ---------------------------------

def ddtm_default_params():
    p = ddtm_params()
    _check(None, _lib.ddtm_default_params(ctypes.byref(p)))
    return p


def ddtm_create(dims, block=None, bc_t=0):
    h = _P()
    d = (_I * 4)(*dims)
    b = (_I * 4)(*block) if block is not None else None
    code = _lib.ddtm_create(ctypes.byref(h), d, b, bc_t)
    if code != OK:
        raise DDTMError(code, "ddtm_create rejected dims=%s block=%s bc_t=%s" % (dims, block, bc_t))
    return h


def ddtm_destroy(ctx):
    _check(None, _lib.ddtm_destroy(ctx))


def ddtm_last_error(ctx):
    return _lib.ddtm_last_error(ctx).decode()


def ddtm_set_stream(ctx, stream_handle):
    _check(ctx, _lib.ddtm_set_stream(ctx, _P(stream_handle)))


def ddtm_get_params(ctx):
    p = ddtm_params()
    _check(ctx, _lib.ddtm_get_params(ctx, ctypes.byref(p)))
    return p


def ddtm_set_params(ctx, p):
    _check(ctx, _lib.ddtm_set_params(ctx, ctypes.byref(p)))


def ddtm_load_gauge(ctx, U, kappa, c_sw):
    pu, loc = _buf(U)
    _check(ctx, _lib.ddtm_load_gauge(ctx, pu, loc, kappa, c_sw))


def ddtm_set_boundary_phases(ctx, theta):
    """Twisted boundary conditions: psi(x + L_mu mu_hat) = exp(i theta[mu]) psi(x), mu = t, x, y, z."""
    t = (_D * 4)(*[float(v) for v in theta])
    _check(ctx, _lib.ddtm_set_boundary_phases(ctx, t))


def ddtm_apply_D(ctx, y, x, nrhs, mu, prec):
    by, bx = _buf(y, True), _buf(x)
    _check(ctx, _lib.ddtm_apply_D(ctx, by[0], bx[0], nrhs, mu, prec, _same_loc(by, bx)))


def ddtm_apply_D_noalloc(ctx, y, x, mu, prec):
    """y = D(mu) x for one right-hand side in device memory, with no allocation
    during the call (fixed scratch inside the library; see include/ddtm.h)."""
    by, bx = _buf(y, True), _buf(x)
    if _same_loc(by, bx) != LOC_DEVICE:
        raise TypeError("ddtm_apply_D_noalloc takes device arrays")
    _check(ctx, _lib.ddtm_apply_D_noalloc(ctx, by[0], bx[0], mu, prec))


def ddtm_sap(ctx, x, b, nrhs, mu, ncycles, nmr, prec):
    bxx, bb = _buf(x, True), _buf(b)
    _check(ctx, _lib.ddtm_sap(ctx, bxx[0], bb[0], nrhs, mu, ncycles, nmr, prec, _same_loc(bxx, bb)))


def ddtm_field_create(ctx, prec, nrhs):
    h = _P()
    _check(ctx, _lib.ddtm_field_create(ctx, prec, nrhs, ctypes.byref(h)))
    return h


def ddtm_field_destroy(f):
    _check(None, _lib.ddtm_field_destroy(f))


def ddtm_field_import(ctx, f, x):
    p, loc = _buf(x)
    _check(ctx, _lib.ddtm_field_import(ctx, f, p, loc))


def ddtm_field_export(ctx, f, x):
    p, loc = _buf(x, True)
    _check(ctx, _lib.ddtm_field_export(ctx, f, p, loc))


def ddtm_apply_D_field(ctx, y, x, mu):
    _check(ctx, _lib.ddtm_apply_D_field(ctx, y, x, mu))


def ddtm_sap_field(ctx, x, b, mu, ncycles, nmr):
    _check(ctx, _lib.ddtm_sap_field(ctx, x, b, mu, ncycles, nmr))


def ddtm_setup(ctx, mu, seed):
    _check(ctx, _lib.ddtm_setup(ctx, mu, seed))


def ddtm_setup_update(ctx, mu, n_iter):
    _check(ctx, _lib.ddtm_setup_update(ctx, mu, n_iter))


def ddtm_set_test_vectors(ctx, level, v, nv):
    p, loc = _buf(v)
    _check(ctx, _lib.ddtm_set_test_vectors(ctx, level, p, nv, loc))


def ddtm_build_coarse(ctx):
    _check(ctx, _lib.ddtm_build_coarse(ctx))


def ddtm_get_prolongator(ctx, level, W):
    p, loc = _buf(W, True)
    _check(ctx, _lib.ddtm_get_prolongator(ctx, level, p, loc))


def ddtm_restrict(ctx, level, c, x, nrhs):
    bc, bx = _buf(c, True), _buf(x)
    _check(ctx, _lib.ddtm_restrict(ctx, level, bc[0], bx[0], nrhs, _same_loc(bc, bx)))


def ddtm_prolong(ctx, level, x, c, nrhs):
    bx, bc = _buf(x, True), _buf(c)
    _check(ctx, _lib.ddtm_prolong(ctx, level, bx[0], bc[0], nrhs, _same_loc(bx, bc)))


def ddtm_apply_Dc(ctx, level, y, x, nrhs, mu):
    by, bx = _buf(y, True), _buf(x)
    _check(ctx, _lib.ddtm_apply_Dc(ctx, level, by[0], bx[0], nrhs, mu, _same_loc(by, bx)))


def ddtm_sap_coarse(ctx, level, x, b, nrhs, mu, ncycles, nmr):
    bxx, bb = _buf(x, True), _buf(b)
    _check(ctx, _lib.ddtm_sap_coarse(ctx, level, bxx[0], bb[0], nrhs, mu, ncycles, nmr, _same_loc(bxx, bb)))


def ddtm_coarse_solve(ctx, x, b, mu_c):
    bxx, bb = _buf(x, True), _buf(b)
    it = _I(0)
    code = _lib.ddtm_coarse_solve(ctx, bxx[0], bb[0], mu_c, _same_loc(bxx, bb), ctypes.byref(it))
    if code not in (OK, ERR_NOCONV):
        _check(ctx, code)
    return it.value, code


def ddtm_coarse_solve_batch(ctx, x, b, nrhs, mu_c):
    bxx, bb = _buf(x, True), _buf(b)
    it = _I(0)
    code = _lib.ddtm_coarse_solve_batch(ctx, bxx[0], bb[0], nrhs, mu_c, _same_loc(bxx, bb), ctypes.byref(it))
    if code not in (OK, ERR_NOCONV):
        _check(ctx, code)
    return it.value, code


def ddtm_solve(ctx, x, b, nrhs, mu):
    bxx, bb = _buf(x, True), _buf(b)
    info = ddtm_solve_info()
    code = _lib.ddtm_solve(ctx, bxx[0], bb[0], nrhs, mu, _same_loc(bxx, bb), ctypes.byref(info))
    if code not in (OK, ERR_NOCONV):
        _check(ctx, code)
    return info, code


def ddtm_eo_cg(ctx, x, b, nrhs, mu, tol=1e-10, max_iter=100000):
    """Even-odd CG baseline (FP64); returns (info, code) like ddtm_solve."""
    bxx, bb = _buf(x, True), _buf(b)
    info = ddtm_solve_info()
    code = _lib.ddtm_eo_cg(ctx, bxx[0], bb[0], nrhs, mu, tol, max_iter, _same_loc(bxx, bb), ctypes.byref(info))
    if code not in (OK, ERR_NOCONV):
        _check(ctx, code)
    return info, code


def ddtm_save_setup(ctx, path):
    _check(ctx, _lib.ddtm_save_setup(ctx, path.encode()))


def ddtm_load_setup(ctx, path):
    _check(ctx, _lib.ddtm_load_setup(ctx, path.encode()))


def ddtm_timer_enable(ctx, on):
    _check(ctx, _lib.ddtm_timer_enable(ctx, 1 if on else 0))


def ddtm_timer_reset(ctx):
    _check(ctx, _lib.ddtm_timer_reset(ctx))


def _timer_json(ctx):
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(ctx, _lib.ddtm_timer_report(ctx, buf, len(buf)))
    return json.loads(buf.value.decode())


def ddtm_timer_report(ctx):
    """Per-kernel {name: {"launches": n, "ms": total, "units": u, "bytes": b}} since the last reset."""
    d = _timer_json(ctx)
    d.pop("_kernel_launches", None)
    return d


def ddtm_timer_kernel_launches(ctx):
    """Kernels the library launched since the last timer reset (timed or not)."""
    return int(_timer_json(ctx).get("_kernel_launches", 0))


def ddtm_measure_fma_peak(prec):
    """(flops per second, best launch ms, SM count) of the SIMT FMA units in FP64 or FP32."""
    f, ms, sms = _D(0), _D(0), _I(0)
    _check(None, _lib.ddtm_measure_fma_peak(prec, ctypes.byref(f), ctypes.byref(ms), ctypes.byref(sms)))
    return f.value, ms.value, sms.value


def ddtm_set_memory_limit(nbytes):
    """Cap the library's device memory (bytes, all contexts); 0 removes the cap."""
    _check(None, _lib.ddtm_set_memory_limit(int(nbytes)))


def ddtm_memory_in_use():
    n = ctypes.c_size_t(0)
    _check(None, _lib.ddtm_memory_in_use(ctypes.byref(n)))
    return n.value


def ddtm_release_workspace(ctx):
    _check(ctx, _lib.ddtm_release_workspace(ctx))


def ddtm_set_option(ctx, name, value):
    _check(ctx, _lib.ddtm_set_option(ctx, name.encode(), int(value)))


def ddtm_get_option(ctx, name):
    v = _I(0)
    _check(ctx, _lib.ddtm_get_option(ctx, name.encode(), ctypes.byref(v)))
    return v.value


def ddtm_autotune_report():
    """{shape: {"ctas_per_sm": k, "ms": [...]}} chosen by the tensor-core pass autotuner so far."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(None, _lib.ddtm_autotune_report(buf, len(buf)))
    return json.loads(buf.value.decode())
