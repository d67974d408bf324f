"""Thin ctypes binding of ``libieti.so`` (argument marshalling only).

Every function has the name of the C entry point it wraps (include/ieti.h).
Device arrays are torch CUDA tensors (FP64, column-major multi-column
vectors are passed as (nrhs, m) row-major tensors, i.e. one contiguous column
per load case); streams are torch.cuda.Stream objects or None. All
computation happens inside the library; there is no CPU fallback: importing
this module fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libieti.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(LIB_PATH)

IETI_OK = 0
IETI_FP64 = 0
IETI_FP32_IR = 1
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "NOT_SIMPLY_CONNECTED", -3: "TREE_INCONSISTENT",
          -4: "SINGULAR_LOCAL", -5: "NO_CONVERGENCE", -6: "TIMEOUT", -7: "CUDA", -8: "OOM",
          -9: "STATE"}


class ieti_problem_desc(C.Structure):
    _fields_ = [("degree", C.c_int), ("npatch", C.c_int * 3), ("nspan_host", C.POINTER(C.c_int) * 3),
                ("periodic0", C.c_int), ("ctrl_host", C.POINTER(C.c_double)),
                ("nu_host", C.POINTER(C.c_double)), ("sub_of_patch_host", C.POINTER(C.c_int)),
                ("source_kind", C.c_int), ("source_params_host", C.POINTER(C.c_double)),
                ("n_source_params", C.c_int), ("nrhs", C.c_int), ("affine", C.c_int)]


class ieti_sizes(C.Structure):
    _fields_ = [("nedge", C.c_int64), ("nnode", C.c_int64), ("n_dirichlet", C.c_int64),
                ("n_tree", C.c_int64), ("n_gauged", C.c_int64), ("m_r", C.c_int64),
                ("n_gp", C.c_int64), ("nsub", C.c_int64), ("nrhs", C.c_int64),
                ("max_nr", C.c_int64), ("max_nI", C.c_int64), ("sum_nr2", C.c_int64),
                ("sum_nI2", C.c_int64), ("bytes_device", C.c_int64), ("tree_rerun", C.c_int)]


class ieti_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinement_steps", C.c_int), ("relres", C.c_double),
                ("global_relres", C.c_double), ("kappa", C.c_double), ("converged", C.c_int),
                ("ms_total", C.c_double), ("fp64_fallback", C.c_int)]


_vp = C.c_void_p
_sig = {
    "ieti_create": (C.c_int, [C.POINTER(ieti_problem_desc), C.POINTER(_vp)]),
    "ieti_create_host": (C.c_int, [C.POINTER(ieti_problem_desc), C.POINTER(_vp)]),
    "ieti_set_params": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]),
    "ieti_assemble": (C.c_int, [_vp, _vp]),
    "ieti_factor": (C.c_int, [_vp, C.c_int, _vp]),
    "ieti_apply_F": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ieti_apply_F_implicit": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ieti_apply_precond": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ieti_solve": (C.c_int, [_vp, _vp, C.c_double, C.c_int, C.c_double, _vp, _vp,
                             C.POINTER(ieti_solve_info), _vp]),
    "ieti_eval_B": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_double), _vp, _vp]),
    "ieti_query": (C.c_int, [_vp, C.POINTER(ieti_sizes)]),
    "ieti_get_dofmap": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_int64,
                                  C.POINTER(C.c_int64)]),
    "ieti_get_block": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int64,
                                 C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ieti_get_coarse": (C.c_int, [_vp, C.POINTER(C.c_double), C.c_int64]),
    "ieti_get_boundary_data": (C.c_int, [_vp, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int64)]),
    "ieti_interface_rhs": (C.c_int, [_vp, _vp, _vp]),
    "ieti_launch_count": (C.c_int64, [_vp]),
    "ieti_debug_set": (C.c_int, [_vp, C.c_int, C.c_int64]),
    "ieti_profile": (C.c_int, [_vp, C.c_int]),
    "ieti_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]),
    "ieti_interface_product_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), _vp, _vp, _vp, C.c_int64, _vp,
                                                 _vp, C.c_int, _vp]),
    "ieti_destroy": (None, [_vp]),
    "ieti_last_error": (C.c_char_p, [_vp]),
    "ieti_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)]),
    "ieti_mlp_query": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "ieti_mlp_set_params": (C.c_int, [_vp, C.POINTER(C.c_float), C.c_int64]),
    "ieti_mlp_set_scaling": (C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float]),
    "ieti_mlp_get": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_int64)]),
    "ieti_mlp_forward": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ieti_mlp_backward": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_float), _vp]),
    "ieti_mlp_adam": (C.c_int, [_vp, C.c_float, _vp]),
    "ieti_mlp_forward_f64": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "ieti_mlp_forward_combine": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, C.c_int, _vp]),
    "ieti_mlp_fit": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_ulonglong,
                               C.c_int, C.POINTER(C.c_float), _vp]),
    "ieti_mlp_destroy": (None, [_vp]),
    "ieti_mlp_last_error": (C.c_char_p, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_symbols():
    """Entry points declared in include/ieti.h."""
    hdr = os.path.join(os.path.dirname(_HERE), "include", "ieti.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(ieti_[a-zA-Z_]+)\s*\(", txt)))


class IetiError(RuntimeError):
    pass


def _check(ctx, st):
    if st != IETI_OK:
        msg = _lib.ieti_last_error(ctx).decode() if ctx else ""
        raise IetiError(f"{STATUS.get(st, st)}: {msg}")


def _dptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(s):
    return C.c_void_p(0 if s is None else s.cuda_stream)


class _Desc:
    """Keeps the host arrays of a descriptor alive for the duration of a call."""

    def __init__(self, prob):
        self.nspan = [np.ascontiguousarray(prob.nspan[d], np.int32) for d in range(3)]
        self.ctrl = np.ascontiguousarray(prob.ctrl, np.float64)
        self.nu = np.ascontiguousarray(prob.nu, np.float64)
        self.sub = np.ascontiguousarray(prob.sub_of_patch, np.int32)
        self.src = np.ascontiguousarray(prob.source_params, np.float64)
        d = ieti_problem_desc()
        d.degree = prob.p
        for i in range(3):
            d.npatch[i] = prob.npatch[i]
            d.nspan_host[i] = self.nspan[i].ctypes.data_as(C.POINTER(C.c_int))
        d.periodic0 = 1 if prob.periodic0 else 0
        d.ctrl_host = self.ctrl.ctypes.data_as(C.POINTER(C.c_double))
        d.nu_host = self.nu.ctypes.data_as(C.POINTER(C.c_double))
        d.sub_of_patch_host = self.sub.ctypes.data_as(C.POINTER(C.c_int))
        d.source_kind = prob.source_kind
        d.source_params_host = self.src.ctypes.data_as(C.POINTER(C.c_double))
        d.n_source_params = len(self.src)
        d.nrhs = prob.nrhs
        d.affine = 1 if prob.affine else 0
        self.desc = d


def ieti_create(prob, host_only=False):
    """Returns an opaque context handle (int)."""
    d = _Desc(prob)
    h = _vp()
    fn = _lib.ieti_create_host if host_only else _lib.ieti_create
    st = fn(C.byref(d.desc), C.byref(h))
    if st != IETI_OK:
        msg = _lib.ieti_last_error(h).decode() if h.value else ""
        if h.value:
            _lib.ieti_destroy(h)
        raise IetiError(f"{STATUS.get(st, st)}: {msg}")
    return h.value


def ieti_create_host(prob):
    return ieti_create(prob, host_only=True)


def ieti_set_params(ctx, nu=None, source_params=None):
    nu_a = None if nu is None else np.ascontiguousarray(nu, np.float64)
    sp_a = None if source_params is None else np.ascontiguousarray(source_params, np.float64)
    _check(ctx, _lib.ieti_set_params(ctx, None if nu_a is None else nu_a.ctypes.data_as(C.POINTER(C.c_double)),
                                     None if sp_a is None else sp_a.ctypes.data_as(C.POINTER(C.c_double)),
                                     0 if sp_a is None else len(sp_a)))


def ieti_assemble(ctx, stream=None):
    _check(ctx, _lib.ieti_assemble(ctx, _stream(stream)))


def ieti_factor(ctx, prec=IETI_FP64, stream=None):
    _check(ctx, _lib.ieti_factor(ctx, int(prec), _stream(stream)))


def ieti_apply_F(ctx, lam, y, nrhs=1, stream=None):
    _check(ctx, _lib.ieti_apply_F(ctx, _dptr(lam), _dptr(y), int(nrhs), _stream(stream)))


def ieti_apply_F_implicit(ctx, lam, y, nrhs=1, stream=None):
    _check(ctx, _lib.ieti_apply_F_implicit(ctx, _dptr(lam), _dptr(y), int(nrhs), _stream(stream)))


def ieti_apply_precond(ctx, r, z, nrhs=1, stream=None):
    _check(ctx, _lib.ieti_apply_precond(ctx, _dptr(r), _dptr(z), int(nrhs), _stream(stream)))


def ieti_solve(ctx, a, lam0=None, tol=1e-8, maxit=500, tol_field=0.0, lam_out=None, stream=None,
               allow_no_convergence=False):
    info = ieti_solve_info()
    st = _lib.ieti_solve(ctx, _dptr(lam0), float(tol), int(maxit), float(tol_field), _dptr(a), _dptr(lam_out),
                         C.byref(info), _stream(stream))
    if not (allow_no_convergence and st == -5):
        _check(ctx, st)
    return info


def ieti_interface_rhs(ctx, b, stream=None):
    _check(ctx, _lib.ieti_interface_rhs(ctx, _dptr(b), _stream(stream)))


IETI_BREF_NONE = 0
IETI_BREF_SINE = 1
IETI_BREF_TRIG = 2


def ieti_eval_B(ctx, a, npatch, nrhs=None, ref_kind=IETI_BREF_NONE, ref_amp=None, B=None, stream=None):
    """a: (nrhs, nedge) float64 CUDA tensor. Returns (nB2, err2) as (nrhs, npatch)
    host arrays of squared L2 norms per patch (err2 is None without a reference);
    B: optional CUDA tensor for the flux at the Gauss points."""
    nr = a.shape[0] if nrhs is None else int(nrhs)
    nB2 = np.zeros(nr * npatch, np.float64)
    err2 = np.zeros(nr * npatch, np.float64) if ref_kind != IETI_BREF_NONE else None
    amp = None if ref_amp is None else np.ascontiguousarray(ref_amp, np.float64)
    _check(ctx, _lib.ieti_eval_B(ctx, _dptr(a), nr, int(ref_kind),
                                 None if amp is None else amp.ctypes.data_as(C.POINTER(C.c_double)),
                                 nB2.ctypes.data_as(C.POINTER(C.c_double)),
                                 None if err2 is None else err2.ctypes.data_as(C.POINTER(C.c_double)),
                                 _dptr(B), _stream(stream)))
    return nB2.reshape(nr, npatch), (None if err2 is None else err2.reshape(nr, npatch))


def ieti_query(ctx):
    s = ieti_sizes()
    _check(ctx, _lib.ieti_query(ctx, C.byref(s)))
    return {f: getattr(s, f) for f, _ in ieti_sizes._fields_}


def ieti_get_dofmap(ctx, which, sub=0):
    n = C.c_int64()
    _check(ctx, _lib.ieti_get_dofmap(ctx, which, sub, None, 0, C.byref(n)))
    out = np.zeros(n.value, np.int64)
    _check(ctx, _lib.ieti_get_dofmap(ctx, which, sub, out.ctypes.data_as(C.POINTER(C.c_int64)), n.value,
                                     C.byref(n)))
    return out


def ieti_get_block(ctx, which, sub):
    R, Cc = C.c_int64(), C.c_int64()
    _check(ctx, _lib.ieti_get_block(ctx, which, sub, None, 0, C.byref(R), C.byref(Cc)))
    out = np.zeros(R.value * Cc.value, np.float64)
    _check(ctx, _lib.ieti_get_block(ctx, which, sub, out.ctypes.data_as(C.POINTER(C.c_double)), len(out),
                                    C.byref(R), C.byref(Cc)))
    return out.reshape(Cc.value, R.value).T


def ieti_get_boundary_data(ctx):
    """Boundary coefficients of IETI_SOURCE_TRIG (nedge values), or an empty array."""
    n = C.c_int64()
    _check(ctx, _lib.ieti_get_boundary_data(ctx, None, 0, C.byref(n)))
    out = np.zeros(n.value, np.float64)
    _check(ctx, _lib.ieti_get_boundary_data(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), n.value,
                                            C.byref(n)))
    return out


def ieti_get_coarse(ctx, n_gp):
    out = np.zeros(n_gp * n_gp, np.float64)
    _check(ctx, _lib.ieti_get_coarse(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), len(out)))
    return out.reshape(n_gp, n_gp).T


def ieti_launch_count(ctx):
    return int(_lib.ieti_launch_count(ctx))


IETI_DEBUG_WAIT_POLLS = 1
IETI_DEBUG_PIVOT_FAULT = 2
IETI_DEBUG_FP64_FALLBACK = 3
IETI_DEBUG_SYRK_TC = 4
IETI_DEBUG_NO_AUTOTUNE = 5
IETI_DEBUG_SYRK_RESERVE = 6
IETI_DEBUG_ELEMENT_LOADS = 7


def ieti_debug_set(ctx, what, value):
    _check(ctx, _lib.ieti_debug_set(ctx, int(what), int(value)))


PROFILE_CLASSES = ["assemble_K", "assemble_j", "potrf_diag", "trsm_panel", "syrk_update", "trsv_fwd",
                   "trsv_bwd", "local_W", "local_S", "gather", "coarse", "pcg_vec", "residual", "other"]


def ieti_profile(ctx, enable=True, classes=None):
    """enable: time every class; classes: names of PROFILE_CLASSES to time alone."""
    if classes is not None:
        mode = sum(2 << PROFILE_CLASSES.index(n) for n in classes)
    else:
        mode = 1 if enable else 0
    _check(ctx, _lib.ieti_profile(ctx, mode))


def ieti_profile_read(ctx):
    n = len(PROFILE_CLASSES)
    ms = (C.c_double * n)()
    calls = (C.c_int64 * n)()
    _check(ctx, _lib.ieti_profile_read(ctx, ms, calls, n))
    return {name: (ms[i], calls[i]) for i, name in enumerate(PROFILE_CLASSES)}


def ieti_interface_product_noalloc(nI, M, dual, weight, x, y, m, nrhs=1, stream=None):
    """y = sum_k B_k^T diag(w_k) M_k diag(w_k) B_k x with the library's fixed scratch.
    nI: host sequence of block sizes; M, dual (int32), weight, x, y: device tensors."""
    nI_a = np.ascontiguousarray(nI, np.int32)
    st = _lib.ieti_interface_product_noalloc(len(nI_a), nI_a.ctypes.data_as(C.POINTER(C.c_int)), _dptr(M),
                                             _dptr(dual), _dptr(weight), int(m), _dptr(x), _dptr(y), int(nrhs),
                                             _stream(stream))
    if st != IETI_OK:
        raise IetiError(f"{STATUS.get(st, st)}: see stderr")


def ieti_destroy(ctx):
    _lib.ieti_destroy(ctx)


def ieti_last_error(ctx):
    return _lib.ieti_last_error(ctx).decode()


# --- learned warm start (3-layer BF16 perceptron) --------------------------------

def _mcheck(m, st):
    if st != IETI_OK:
        msg = _lib.ieti_mlp_last_error(m).decode() if m else ""
        raise IetiError(f"{STATUS.get(st, st)}: {msg}")


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def ieti_mlp_create(n_in, n_hidden, n_out, max_batch):
    m = C.c_void_p()
    st = _lib.ieti_mlp_create(int(n_in), int(n_hidden), int(n_out), int(max_batch), C.byref(m))
    if st != IETI_OK:
        if m:
            _lib.ieti_mlp_destroy(m)
        _mcheck(None, st)
    return m


def ieti_mlp_query(m):
    sz = (C.c_int * 4)()
    npar = C.c_int64()
    _mcheck(m, _lib.ieti_mlp_query(m, sz, C.byref(npar)))
    return {"n_in": sz[0], "n_hidden": sz[1], "n_out": sz[2], "max_batch": sz[3], "nparam": npar.value}


def ieti_mlp_set_params(m, params):
    """params: flat host vector W1|b1|W2|b2|W3|b3 (or a list of those arrays)."""
    if isinstance(params, (list, tuple)):
        params = np.concatenate([np.ravel(p) for p in params])
    p = _f32(params)
    _mcheck(m, _lib.ieti_mlp_set_params(m, p.ctypes.data_as(C.POINTER(C.c_float)), p.size))


def ieti_mlp_set_scaling(m, shift, scale, out_scale=1.0):
    a, b = _f32(shift), _f32(scale)
    _mcheck(m, _lib.ieti_mlp_set_scaling(m, a.ctypes.data_as(C.POINTER(C.c_float)),
                                         b.ctypes.data_as(C.POINTER(C.c_float)), float(out_scale)))


def ieti_mlp_get(m, which=0):
    n = C.c_int64()
    _mcheck(m, _lib.ieti_mlp_get(m, int(which), None, 0, C.byref(n)))
    out = np.empty(n.value, np.float32)
    _mcheck(m, _lib.ieti_mlp_get(m, int(which), out.ctypes.data_as(C.POINTER(C.c_float)), n.value, C.byref(n)))
    return out


def ieti_mlp_forward(m, x, y, batch=None, stream=None):
    """x: (batch, n_in) float32 CUDA tensor; y: (batch, n_out) float32 CUDA tensor."""
    b = x.shape[0] if batch is None else batch
    _mcheck(m, _lib.ieti_mlp_forward(m, _dptr(x), _dptr(y), int(b), _stream(stream)))


def ieti_mlp_forward_f64(m, x, lam, batch=None, stream=None):
    """lam: (batch, n_out) float64 CUDA tensor (the lam0 layout of ieti_solve)."""
    b = x.shape[0] if batch is None else batch
    _mcheck(m, _lib.ieti_mlp_forward_f64(m, _dptr(x), _dptr(lam), int(b), _stream(stream)))


def ieti_mlp_forward_combine(m, x, coef, lam, batch=None, stream=None):
    """x (batch, n_in) float32, coef (batch, ncoef) float64, lam (batch, n_out/ncoef)
    float64: CUDA tensors."""
    b = x.shape[0] if batch is None else batch
    _mcheck(m, _lib.ieti_mlp_forward_combine(m, _dptr(x), _dptr(coef), int(coef.shape[1]), _dptr(lam), int(b),
                                             _stream(stream)))


def ieti_mlp_fit(m, X, T, batch, epochs, lr, decay=1.0, seed=0, normalise=True, stream=None):
    """Trains on all rows of X (n, n_in) / T (n, n_out), float32 CUDA tensors;
    returns the mean batch loss of the last epoch."""
    loss = C.c_float(float("nan"))
    _mcheck(m, _lib.ieti_mlp_fit(m, _dptr(X), _dptr(T), int(X.shape[0]), int(batch), int(epochs), float(lr),
                                 float(decay), int(seed), int(bool(normalise)), C.byref(loss), _stream(stream)))
    return loss.value


def ieti_mlp_backward(m, x, t, batch=None, want_loss=True, stream=None):
    b = x.shape[0] if batch is None else batch
    loss = C.c_float(float("nan"))
    _mcheck(m, _lib.ieti_mlp_backward(m, _dptr(x), _dptr(t), int(b), C.byref(loss) if want_loss else None,
                                      _stream(stream)))
    return loss.value if want_loss else None


def ieti_mlp_adam(m, lr, stream=None):
    _mcheck(m, _lib.ieti_mlp_adam(m, float(lr), _stream(stream)))


def ieti_mlp_destroy(m):
    _lib.ieti_mlp_destroy(m)


def ieti_mlp_last_error(m):
    return _lib.ieti_mlp_last_error(m).decode()
