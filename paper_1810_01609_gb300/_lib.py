"""ctypes binding of libmdwf (include/mdwf.h): same names, argument marshalling only.

Every function raises MdwfError (with the C status in .code) when the C call fails and
returns the call's outputs otherwise.  Array arguments may be torch tensors (device
pointers) or numpy arrays (host pointers); `where` is derived from them.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmdwf.so")

MDWF_SUCCESS = 0
MDWF_ERR_ARG = -1
MDWF_ERR_CUDA = -2
MDWF_ERR_OOM = -3
MDWF_ERR_NOT_SU3 = -4
MDWF_ERR_NOT_CONVERGED = -5
MDWF_ERR_BREAKDOWN = -6
MDWF_ERR_TIMEOUT = -7
MDWF_ERR_STATE = -8

MDWF_PREC_F64, MDWF_PREC_F32, MDWF_PREC_F16, MDWF_PREC_BF16, MDWF_PREC_I16 = 0, 1, 2, 3, 4
PRECS = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "i16": 4, "f64e": 5}   # f64e: mdwf_apply only
MDWF_HOST, MDWF_DEVICE = 0, 1
MDWF_PC_LEFT, MDWF_PC_SYM = 0, 1
PC_FORMS = {"left": 0, "sym": 1}
OPS = ["HOP_EO", "HOP_OE", "HOP_EO_DAG", "HOP_OE_DAG", "D5", "D5_DAG", "M5", "M5_DAG", "M5INV",
       "M5INV_DAG", "HOP_EO_M5INV", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "FULL_D", "FULL_D_DAG",
       "MPC_SYM", "MPC_SYM_DAG"]
OP = {n: i for i, n in enumerate(OPS)}


class mdwf_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("Ls", ctypes.c_int), ("b5", ctypes.c_double),
                ("c5", ctypes.c_double), ("M5", ctypes.c_double), ("mf", ctypes.c_double),
                ("t_bc", ctypes.c_double), ("gauge_recon", ctypes.c_int), ("check_su3", ctypes.c_int),
                ("t_ranks", ctypes.c_int), ("t_rank", ctypes.c_int), ("f64_emulation", ctypes.c_int)]


class mdwf_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("sloppy_prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("ru_interval", ctypes.c_int), ("check_interval", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("location", ctypes.c_int), ("full_residual", ctypes.c_int),
                ("pc_form", ctypes.c_int)]


class mdwf_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("full_residual", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("fp64_residuals", ctypes.c_int),
                ("emulated_residuals", ctypes.c_int)]


class MdwfError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s (%d): %s" % (strerror(code) if _lib else "error", code, what))


_lib = None
_V, _I, _D, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
# int (*)(void* user, const void* send_lo, const void* send_hi, void* recv_lo, void* recv_hi, size_t, void* stream)
FACE_EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, _V, _V, _V, _V, _V, _S, _V)
_SIGS = {
    "mdwf_default_params": (None, [ctypes.POINTER(mdwf_params)]),
    "mdwf_default_solve_params": (None, [ctypes.POINTER(mdwf_solve_params)]),
    "mdwf_create": (_I, [ctypes.POINTER(mdwf_params), ctypes.POINTER(_V)]),
    "mdwf_destroy": (None, [_V]),
    "mdwf_load_gauge": (_I, [_V, _V, _I, _V]),
    "mdwf_field_bytes": (_I, [_V, _I, _I, ctypes.POINTER(_S)]),
    "mdwf_pack": (_I, [_V, _V, _V, _I, _I, _V]),
    "mdwf_unpack": (_I, [_V, _V, _V, _I, _I, _V]),
    "mdwf_apply": (_I, [_V, _I, _I, _V, _V, _I, _V]),
    "mdwf_solve": (_I, [_V, _V, _V, ctypes.POINTER(mdwf_solve_params), ctypes.POINTER(mdwf_solve_info), _V]),
    "mdwf_solve_multi": (_I, [_V, _I, _V, _V, ctypes.POINTER(mdwf_solve_params),
                              ctypes.POINTER(mdwf_solve_info), _V]),
    "mdwf_make_source_4d": (_I, [_V, _V, _V, _I, _I, _V]),
    "mdwf_propagator": (_I, [_V, _I, _V, _V, _I, ctypes.POINTER(mdwf_solve_params),
                             ctypes.POINTER(mdwf_solve_info), _V]),
    "mdwf_project_4d": (_I, [_V, _V, _V, _I, _I, _V]),
    "mdwf_fh_source": (_I, [_V, _V, _V, _I, _I, _V]),
    "mdwf_contract_nucleon": (_I, [_V, _V, _V, _V, _V, _I, _V]),
    "mdwf_contract_nucleon_noalloc": (_I, [_V, _V, _V, _V, _V, _V]),
    "mdwf_noalloc_last_error": (ctypes.c_char_p, []),
    "mdwf_fh_effective_coupling": (_I, [_V, _V, _V, _I]),
    "mdwf_set_tuning": (_I, [_V, _I]),
    "mdwf_tune_entries": (_I, [_V, ctypes.POINTER(_I)]),
    "mdwf_tune_entry": (_I, [_V, _I, ctypes.c_char_p, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "mdwf_launch_count": (ctypes.c_longlong, [_V]),
    "mdwf_algorithmic_bytes": (ctypes.c_double, [_V]),
    "mdwf_set_face_exchange": (_I, [_V, FACE_EXCHANGE_FN, _V]),
    "mdwf_face_bytes": (_I, [_V, _I, _I, ctypes.POINTER(_S)]),
    "mdwf_set_face_buffers": (_I, [_V, _V, _V, _V, _V, _S]),
    "mdwf_group_partitions": (_I, [ctypes.POINTER(_V), _I]),
    "mdwf_strerror": (ctypes.c_char_p, [_I]),
    "mdwf_last_error": (ctypes.c_char_p, []),
}


def load():
    """Load libmdwf.so (fails loudly if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmdwf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(code):
    if code != MDWF_SUCCESS:
        raise MdwfError(code, load().mdwf_last_error().decode())
    return code


def strerror(code):
    return load().mdwf_strerror(code).decode()


def ptr(a):
    """(address, location) of a torch tensor or numpy array."""
    if a is None:
        return None, MDWF_DEVICE
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return a.ctypes.data, MDWF_HOST
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), (MDWF_DEVICE if a.is_cuda else MDWF_HOST)


def _stream(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def mdwf_default_params():
    p = mdwf_params()
    load().mdwf_default_params(ctypes.byref(p))
    return p


def mdwf_default_solve_params():
    sp = mdwf_solve_params()
    load().mdwf_default_solve_params(ctypes.byref(sp))
    return sp


def mdwf_create(params):
    h = ctypes.c_void_p()
    _check(load().mdwf_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def mdwf_destroy(ctx):
    load().mdwf_destroy(ctx)


def mdwf_load_gauge(ctx, links, stream=None):
    p, where = ptr(links)
    return _check(load().mdwf_load_gauge(ctx, p, where, _stream(stream)))


def mdwf_field_bytes(ctx, prec, nrhs):
    n = ctypes.c_size_t()
    _check(load().mdwf_field_bytes(ctx, prec, nrhs, ctypes.byref(n)))
    return n.value


def mdwf_pack(ctx, user5d, internal, prec, nrhs, stream=None):
    return _check(load().mdwf_pack(ctx, ptr(user5d)[0], ptr(internal)[0], prec, nrhs, _stream(stream)))


def mdwf_unpack(ctx, internal, user5d, prec, nrhs, stream=None):
    return _check(load().mdwf_unpack(ctx, ptr(internal)[0], ptr(user5d)[0], prec, nrhs, _stream(stream)))


def mdwf_apply(ctx, op, prec, inp, out, nrhs, stream=None):
    return _check(load().mdwf_apply(ctx, op, prec, ptr(inp)[0], ptr(out)[0], nrhs, _stream(stream)))


def mdwf_solve(ctx, src, sol, sp, stream=None):
    info = mdwf_solve_info()
    code = load().mdwf_solve(ctx, ptr(src)[0], ptr(sol)[0], ctypes.byref(sp), ctypes.byref(info), _stream(stream))
    if code not in (MDWF_SUCCESS, MDWF_ERR_NOT_CONVERGED):
        _check(code)
    return info


def mdwf_solve_multi(ctx, nrhs, src, sol, sp, stream=None):
    infos = (mdwf_solve_info * nrhs)()
    code = load().mdwf_solve_multi(ctx, nrhs, ptr(src)[0], ptr(sol)[0], ctypes.byref(sp), infos, _stream(stream))
    if code not in (MDWF_SUCCESS, MDWF_ERR_NOT_CONVERGED):
        _check(code)
    return list(infos)


def _io4(fn, ctx, a, b, nrhs, stream):
    pa, wa = ptr(a)
    pb, wb = ptr(b)
    if wa != wb:
        raise ValueError("input and output must both be host or both be device arrays")
    return _check(fn(ctx, pa, pb, nrhs, wa, _stream(stream)))


def mdwf_propagator(ctx, nrhs, src4d, q4d, sp, stream=None):
    """4D sources -> 4D propagator columns in one call (host or device arrays, both alike)."""
    pa, wa = ptr(src4d)
    pb, wb = ptr(q4d)
    if wa != wb:
        raise ValueError("source and propagator must both be host or both be device arrays")
    infos = (mdwf_solve_info * nrhs)()
    code = load().mdwf_propagator(ctx, nrhs, pa, pb, wa, ctypes.byref(sp), infos, _stream(stream))
    if code not in (MDWF_SUCCESS, MDWF_ERR_NOT_CONVERGED):
        _check(code)
    return list(infos)


def mdwf_make_source_4d(ctx, src4d, src5d, nrhs, stream=None):
    return _io4(load().mdwf_make_source_4d, ctx, src4d, src5d, nrhs, stream)


def mdwf_project_4d(ctx, sol5d, q4d, nrhs, stream=None):
    return _io4(load().mdwf_project_4d, ctx, sol5d, q4d, nrhs, stream)


def mdwf_fh_source(ctx, q4d, out4d, nrhs, stream=None):
    return _io4(load().mdwf_fh_source, ctx, q4d, out4d, nrhs, stream)


def mdwf_contract_nucleon(ctx, u1, d, u2, corr, stream=None):
    ps = [ptr(x) for x in (u1, d, u2, corr)]
    wheres = {w for _, w in ps}
    if len(wheres) != 1:
        raise ValueError("all arrays must be host or all device")
    return _check(load().mdwf_contract_nucleon(ctx, ps[0][0], ps[1][0], ps[2][0], ps[3][0], wheres.pop(),
                                               _stream(stream)))


def mdwf_contract_nucleon_noalloc(ctx, u1, d, u2, corr, stream=None):
    """Allocation-free contraction (device arrays only); see include/mdwf.h."""
    ps = [ptr(x) for x in (u1, d, u2, corr)]
    if any(w != MDWF_DEVICE for _, w in ps):
        raise ValueError("mdwf_contract_nucleon_noalloc takes device arrays only")
    code = load().mdwf_contract_nucleon_noalloc(ctx, ps[0][0], ps[1][0], ps[2][0], ps[3][0], _stream(stream))
    if code != MDWF_SUCCESS:
        raise MdwfError(code, load().mdwf_noalloc_last_error().decode())
    return code


def mdwf_set_tuning(ctx, enable):
    return _check(load().mdwf_set_tuning(ctx, int(enable)))


def mdwf_tune_entries(ctx):
    n = ctypes.c_int()
    _check(load().mdwf_tune_entries(ctx, ctypes.byref(n)))
    out = []
    for i in range(n.value):
        key = ctypes.create_string_buffer(512)
        ns = ctypes.c_int()
        ms = ctypes.c_double()
        _check(load().mdwf_tune_entry(ctx, i, key, 512, ctypes.byref(ns), ctypes.byref(ms)))
        out.append((key.value.decode(), ns.value, ms.value))
    return out


def mdwf_launch_count(ctx):
    return load().mdwf_launch_count(ctx)


def mdwf_algorithmic_bytes(ctx):
    return load().mdwf_algorithmic_bytes(ctx)


def mdwf_last_error():
    return load().mdwf_last_error().decode()


def mdwf_set_face_exchange(ctx, fn, user=None):
    """fn: a FACE_EXCHANGE_FN (keep a reference to it while the context uses it) or None."""
    return _check(load().mdwf_set_face_exchange(ctx, fn if fn is not None else FACE_EXCHANGE_FN(), user))


def mdwf_face_bytes(ctx, prec, nrhs):
    n = ctypes.c_size_t()
    _check(load().mdwf_face_bytes(ctx, prec, nrhs, ctypes.byref(n)))
    return n.value


def mdwf_set_face_buffers(ctx, send_lo, send_hi, recv_lo, recv_hi, nbytes):
    ps = [ptr(x)[0] if x is not None else None for x in (send_lo, send_hi, recv_lo, recv_hi)]
    return _check(load().mdwf_set_face_buffers(ctx, ps[0], ps[1], ps[2], ps[3], nbytes))


def mdwf_group_partitions(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    return _check(load().mdwf_group_partitions(arr, len(ctxs)))


def mdwf_fh_effective_coupling(c2, c3):
    """c2 = C(t), c3 = C_FH(t): T complex values (numpy or torch); returns geff (T - 1)."""
    a = np.ascontiguousarray(np.asarray(c2.cpu() if hasattr(c2, "cpu") else c2, dtype=np.complex128))
    b = np.ascontiguousarray(np.asarray(c3.cpu() if hasattr(c3, "cpu") else c3, dtype=np.complex128))
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("c2 and c3 must be 1-D of the same length")
    out = np.empty(a.shape[0] - 1, dtype=np.float64)
    _check(load().mdwf_fh_effective_coupling(a.ctypes.data, b.ctypes.data, out.ctypes.data, a.shape[0]))
    return out
