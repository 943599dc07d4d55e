"""ctypes binding of the C-ABI in include/sapmg.h (argument marshalling only).

Every function here has the name of the C entry point it calls and takes the
same arguments, with torch tensors accepted wherever the C side takes a device
pointer.  All computation happens in libsapmg.so; if the library is missing or
cannot be loaded the first call raises, there is no fallback.  With
SAPMG_LIBRARY=debug in the environment the binding loads libsapmg_debug.so,
the build with device-side index checks (mg_debug_failures).
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsapmg_debug.so" if os.environ.get("SAPMG_LIBRARY") == "debug"
                        else "libsapmg.so")

MG_OK = 0
MG_NOT_CONVERGED = 1
MG_ERR_ARG = -1
MG_ERR_NONFINITE = -2
MG_ERR_OOM = -3
MG_ERR_CUDA = -4
MG_ERR_TIMEOUT = -5
MG_ERR_STATE = -6
MG_ERR_BOUNDS = -7

MG_FP64 = 0
MG_FP32 = 1
MG_FP16 = 2
MG_BF16 = 3
MG_BLOCKED = 0x100
MG_DAGGER = 0x200
MG_FP64_ON_FP32 = 0x400

PRECISIONS = {"fp64": MG_FP64, "fp32": MG_FP32, "fp16": MG_FP16, "bf16": MG_BF16}


class MgParams(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 4),
        ("antiperiodic_t", ctypes.c_int),
        ("n_levels", ctypes.c_int),
        ("agg2", ctypes.c_int * 4),
        ("sap_block2", ctypes.c_int * 4),
        ("n_vec", ctypes.c_int * 2),
        ("setup_iters", ctypes.c_int),
        ("n_mr", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("coarse_iters", ctypes.c_int),
        ("inner_iters", ctypes.c_int),
        ("fgmres_m", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("maxiter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nrhs_max", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("stream", ctypes.c_void_p),
        ("init_vectors", ctypes.c_void_p),
        ("verbose", ctypes.c_int),
        ("setup2_iters", ctypes.c_int),
        ("setup2_start", ctypes.c_void_p),
        ("autotune", ctypes.c_int),
        ("init_vectors_prec", ctypes.c_int),
    ]


class MgSolveInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("relres", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("precond_seconds", ctypes.c_double),
    ]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_SIGNATURES = {
    "mg_default_params": (_I, [ctypes.POINTER(MgParams)]),
    "mg_setup": (_I, [_VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(MgParams), ctypes.POINTER(_VP)]),
    "dirac_apply": (_I, [_VP, _VP, _VP, _I, _I]),
    "sap_smooth": (_I, [_VP, _VP, _VP, _I, _I, _I]),
    "mg_solve": (_I, [_VP, _VP, _VP, _I, ctypes.POINTER(MgSolveInfo)]),
    "mg_cgn_solve": (_I, [_VP, _VP, _VP, _I, _I, ctypes.c_double, _I, ctypes.POINTER(MgSolveInfo)]),
    "mg_harmonic_ritz": (_I, [_I, _VP, _VP, _VP]),
    "mg_eigh": (_I, [_I, _VP, _VP, _VP]),
    "mg_destroy": (None, [_VP]),
    "mg_save": (_I, [_VP, ctypes.c_char_p]),
    "mg_setup_load": (_I, [_VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(MgParams), ctypes.c_char_p,
                           ctypes.POINTER(_VP)]),
    "mg_last_error": (ctypes.c_char_p, []),
    "mg_sizeof_params": (ctypes.c_ulong, []),
    "mg_pack_spinor": (_I, [_VP, _VP, _VP, _I, _I]),
    "mg_unpack_spinor": (_I, [_VP, _VP, _VP, _I, _I]),
    "mg_clover_export": (_I, [_VP, _VP]),
    "mg_get_vectors": (_I, [_VP, _I, _VP]),
    "mg_get_coarse_op": (_I, [_VP, _I, _VP]),
    "mg_restrict": (_I, [_VP, _I, _VP, _VP, _I]),
    "mg_prolong": (_I, [_VP, _I, _VP, _VP, _I]),
    "mg_coarse_apply": (_I, [_VP, _I, _VP, _VP, _I]),
    "mg_coarse_apply_batch": (_I, [_VP, _I, _VP, _VP, _I, _I]),
    "mg_restrict_batch": (_I, [_VP, _I, _VP, _VP, _I, _I]),
    "mg_prolong_batch": (_I, [_VP, _I, _VP, _VP, _I, _I]),
    "mg_coarse_solve": (_I, [_VP, _I, _VP, _VP, _I]),
    "mg_coarse_solve_noalloc": (_I, [_VP, _I, _VP, _VP, _I]),
    "mg_precondition": (_I, [_VP, _VP, _VP, _I]),
    "mg_set_profiling": (_I, [_VP, _I]),
    "mg_get_profile": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    "mg_get_profile_bytes": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_double)]),
    "mg_reset_profile": (_I, [_VP]),
    "mg_launch_count": (ctypes.c_longlong, []),
    "mg_sync": (_I, [_VP]),
    "mg_debug_failures": (ctypes.c_longlong, []),
    "mg_debug_check": (_I, [ctypes.c_longlong, ctypes.c_longlong]),
    "mg_get_history": (_I, [_VP, _VP, _I]),
    "mg_get_tuning": (_I, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "mg_set_wait_limit": (_I, [_VP, _I]),
    "mg_probe_peaks": (_I, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)]),
    "mg_net_layer_forward": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "mg_net_layer_forward_bf16": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "mg_net_layer_backward": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP]),
    "mg_net_gate_forward": (_I, [_VP, _I, _VP, _VP]),
    "mg_net_gate_backward": (_I, [_VP, _I, _VP, _VP, _VP]),
    "mg_net_loss": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "mg_adam_step": (_I, [_VP, ctypes.c_size_t, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, ctypes.c_double, _I]),
}

_lib = None


def lib():
    """The loaded libsapmg.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build(), the "
                               "MG_DEBUG variant with python -m paper_1202_2462_gb300._build --debug "
                               "(there is no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        if handle.mg_sizeof_params() != ctypes.sizeof(MgParams):
            raise RuntimeError("mg_params layout mismatch between binding and library")
        _lib = handle
    return _lib


class MgError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().mg_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(code, where):
    if code < 0:
        raise MgError(code, where)
    return code


# --- entry points with the C names ---------------------------------------------

def mg_default_params():
    p = MgParams()
    _check(lib().mg_default_params(ctypes.byref(p)), "mg_default_params")
    return p


def mg_setup(U, c_sw, m0, params):
    ctx = ctypes.c_void_p()
    _check(lib().mg_setup(_ptr(U), float(c_sw), float(m0), ctypes.byref(params), ctypes.byref(ctx)), "mg_setup")
    return ctx


def mg_save(ctx, path):
    return _check(lib().mg_save(ctx, os.fsencode(path)), "mg_save")


def mg_setup_load(U, c_sw, m0, params, path):
    """A context whose test vectors come from a file written by mg_save."""
    ctx = _VP()
    _check(lib().mg_setup_load(_ptr(U), float(c_sw), float(m0), ctypes.byref(params), os.fsencode(path),
                               ctypes.byref(ctx)), "mg_setup_load")
    return ctx


def dirac_apply(ctx, inp, out, prec, nrhs=1):
    return _check(lib().dirac_apply(ctx, _ptr(inp), _ptr(out), prec, nrhs), "dirac_apply")


def sap_smooth(ctx, b, z, n_sweeps, prec, nrhs=1):
    return _check(lib().sap_smooth(ctx, _ptr(b), _ptr(z), n_sweeps, prec, nrhs), "sap_smooth")


def mg_solve(ctx, b, z, nrhs=1):
    info = MgSolveInfo()
    code = _check(lib().mg_solve(ctx, _ptr(b), _ptr(z), nrhs, ctypes.byref(info)), "mg_solve")
    return code, info


def mg_cgn_solve(ctx, b, z, nrhs, prec, tol, maxiter):
    info = MgSolveInfo()
    code = _check(lib().mg_cgn_solve(ctx, _ptr(b), _ptr(z), nrhs, prec, float(tol), int(maxiter), ctypes.byref(info)),
                  "mg_cgn_solve")
    return code, info


def mg_harmonic_ritz(hbar):
    """(m+1) x m complex numpy Hessenberg matrix -> (theta (m,), y (m, m)), host only."""
    import numpy as np
    m = hbar.shape[1]
    h = np.asfortranarray(hbar, dtype=np.complex128)
    theta = np.zeros(m, dtype=np.complex128)
    y = np.zeros((m, m), dtype=np.complex128, order="F")
    _check(lib().mg_harmonic_ritz(m, h.ctypes.data, theta.ctypes.data, y.ctypes.data), "mg_harmonic_ritz")
    return theta, y


def mg_eigh(a):
    """Hermitian complex numpy matrix -> (ascending eigenvalues, eigenvectors as columns), host only."""
    import numpy as np
    n = a.shape[0]
    am = np.asfortranarray(a, dtype=np.complex128)
    w = np.zeros(n, dtype=np.float64)
    v = np.zeros((n, n), dtype=np.complex128, order="F")
    _check(lib().mg_eigh(n, am.ctypes.data, w.ctypes.data, v.ctypes.data), "mg_eigh")
    return w, v


def mg_destroy(ctx):
    lib().mg_destroy(ctx)


def mg_pack_spinor(ctx, canonical, blocked, prec, nrhs=1):
    return _check(lib().mg_pack_spinor(ctx, _ptr(canonical), _ptr(blocked), prec, nrhs), "mg_pack_spinor")


def mg_unpack_spinor(ctx, blocked, canonical, prec, nrhs=1):
    return _check(lib().mg_unpack_spinor(ctx, _ptr(blocked), _ptr(canonical), prec, nrhs), "mg_unpack_spinor")


def mg_clover_export(ctx, out):
    return _check(lib().mg_clover_export(ctx, _ptr(out)), "mg_clover_export")


def mg_get_vectors(ctx, level, out):
    return _check(lib().mg_get_vectors(ctx, level, _ptr(out)), "mg_get_vectors")


def mg_get_coarse_op(ctx, level, out):
    return _check(lib().mg_get_coarse_op(ctx, level, _ptr(out)), "mg_get_coarse_op")


def mg_restrict(ctx, level, inp, out, prec):
    return _check(lib().mg_restrict(ctx, level, _ptr(inp), _ptr(out), prec), "mg_restrict")


def mg_prolong(ctx, level, inp, out, prec):
    return _check(lib().mg_prolong(ctx, level, _ptr(inp), _ptr(out), prec), "mg_prolong")


def mg_coarse_apply(ctx, level, inp, out, prec):
    return _check(lib().mg_coarse_apply(ctx, level, _ptr(inp), _ptr(out), prec), "mg_coarse_apply")


def mg_restrict_batch(ctx, level, inp, out, prec, nrhs):
    return _check(lib().mg_restrict_batch(ctx, level, _ptr(inp), _ptr(out), prec, nrhs), "mg_restrict_batch")


def mg_prolong_batch(ctx, level, inp, out, prec, nrhs):
    return _check(lib().mg_prolong_batch(ctx, level, _ptr(inp), _ptr(out), prec, nrhs), "mg_prolong_batch")


def mg_coarse_apply_batch(ctx, level, inp, out, prec, nrhs):
    return _check(lib().mg_coarse_apply_batch(ctx, level, _ptr(inp), _ptr(out), prec, nrhs), "mg_coarse_apply_batch")


def mg_coarse_solve(ctx, level, inp, out, prec):
    return _check(lib().mg_coarse_solve(ctx, level, _ptr(inp), _ptr(out), prec), "mg_coarse_solve")


def mg_coarse_solve_noalloc(ctx, level, inp, out, prec):
    return _check(lib().mg_coarse_solve_noalloc(ctx, level, _ptr(inp), _ptr(out), prec), "mg_coarse_solve_noalloc")


def mg_precondition(ctx, v, z, prec):
    return _check(lib().mg_precondition(ctx, _ptr(v), _ptr(z), prec), "mg_precondition")


def mg_set_profiling(ctx, on):
    return _check(lib().mg_set_profiling(ctx, int(on)), "mg_set_profiling")


def mg_get_profile(ctx, family):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(lib().mg_get_profile(ctx, family, ctypes.byref(n), ctypes.byref(ms)), "mg_get_profile")
    return n.value, ms.value


def mg_get_profile_bytes(ctx, family):
    b = ctypes.c_double()
    _check(lib().mg_get_profile_bytes(ctx, family, ctypes.byref(b)), "mg_get_profile_bytes")
    return b.value


def mg_net_layer_forward(ctx, cin, cout, w, x, y):
    return _check(lib().mg_net_layer_forward(ctx, cin, cout, _ptr(w), _ptr(x), _ptr(y)), "mg_net_layer_forward")


def mg_net_layer_forward_bf16(ctx, cin, cout, W, x, y):
    """W: a device tensor of BF16 (re, im) pairs [cout][cin][9][4][4][2]."""
    return _check(lib().mg_net_layer_forward_bf16(ctx, cin, cout, _ptr(W), _ptr(x), _ptr(y)),
                  "mg_net_layer_forward_bf16")


def mg_net_layer_backward(ctx, cin, cout, w, x, gy, gx, gw):
    return _check(lib().mg_net_layer_backward(ctx, cin, cout, _ptr(w), _ptr(x), _ptr(gy), _ptr(gx), _ptr(gw)),
                  "mg_net_layer_backward")


def mg_net_gate_forward(ctx, channels, x, y):
    return _check(lib().mg_net_gate_forward(ctx, channels, _ptr(x), _ptr(y)), "mg_net_gate_forward")


def mg_net_gate_backward(ctx, channels, x, gy, gx):
    return _check(lib().mg_net_gate_backward(ctx, channels, _ptr(x), _ptr(gy), _ptr(gx)), "mg_net_gate_backward")


def mg_net_loss(ctx, y, t, gy):
    out = ctypes.c_double()
    _check(lib().mg_net_loss(ctx, _ptr(y), _ptr(t), _ptr(gy), ctypes.byref(out)), "mg_net_loss")
    return out.value


def mg_adam_step(ctx, n, p, g, m, v, lr, beta1, beta2, eps, step):
    return _check(lib().mg_adam_step(ctx, n, _ptr(p), _ptr(g), _ptr(m), _ptr(v), lr, beta1, beta2, eps, step),
                  "mg_adam_step")


def mg_reset_profile(ctx):
    return _check(lib().mg_reset_profile(ctx), "mg_reset_profile")


def mg_launch_count():
    return lib().mg_launch_count()


def mg_get_tuning(ctx):
    """The context's launch shapes (see include/sapmg.h): a dict."""
    a = (ctypes.c_int * 6)()
    _check(lib().mg_get_tuning(ctx, a), "mg_get_tuning")
    return {"source": ("default", "tuned", "cached")[a[0]], "sap_shape": a[1], "xfer_batch": a[2],
            "coarse_stages": a[3], "coarse_ctas_per_sm": a[4], "coarse_batch": a[5]}


def mg_get_history(ctx):
    """The last solve's residual history: a list of (iteration, rhs, relative residual)."""
    n = _check(lib().mg_get_history(ctx, None, 0), "mg_get_history")
    buf = (ctypes.c_double * (3 * max(n, 1)))()
    _check(lib().mg_get_history(ctx, buf, n), "mg_get_history")
    return [(int(buf[3 * k]), int(buf[3 * k + 1]), buf[3 * k + 2]) for k in range(n)]


def mg_sync(ctx):
    return _check(lib().mg_sync(ctx), "mg_sync")


def mg_debug_failures():
    """Failed device-side index checks since the previous call (MG_DEBUG
    build), or -1 for the release build."""
    n = lib().mg_debug_failures()
    return _check(n, "mg_debug_failures") if n < -1 else n


def mg_debug_check(value, bound):
    return _check(lib().mg_debug_check(value, bound), "mg_debug_check")


def mg_set_wait_limit(ctx, spins):
    return _check(lib().mg_set_wait_limit(ctx, spins), "mg_set_wait_limit")


def mg_probe_peaks(stream=None):
    """(FP32 TFLOP/s scalar FMA, FP32 TFLOP/s packed FMA, shared-memory GB/s) of the current device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    s = ctypes.c_void_p(stream.cuda_stream if stream is not None else None)
    _check(lib().mg_probe_peaks(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "mg_probe_peaks")
    return a.value, b.value, c.value


def profile_mask(*families):
    """mg_set_profiling mask selecting the named families."""
    m = 0
    for f in families:
        m |= 1 << (PROFILE_FAMILIES[f] + 1)
    return m


PROFILE_FAMILIES = {"dirac": 0, "sap": 1, "coarse": 2, "restrict": 3, "prolong": 4, "blas": 5, "coarse_blas": 6,
                    "sap1": 7}
