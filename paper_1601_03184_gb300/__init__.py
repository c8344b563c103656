"""GB300 (sm_103a) multiple-right-hand-side setup of two-level DD-alpha-AMG
for the Wilson-clover Dirac operator (arXiv:1601.03184).

This module is a thin ctypes binding of the C ABI declared in include/mrhs.h.
Every function named mrhs_* here has the same name, arguments and meaning as
its C counterpart; it only marshals arguments (numpy arrays -> host pointers,
torch CUDA tensors -> device pointers) and raises MrhsError on a non-zero
status. All computation happens in libmrhs.so's CUDA kernels; there is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrhs.so")

# enums of mrhs.h
MRHS_OK = 0
MRHS_ERR_ARG, MRHS_ERR_SHAPE, MRHS_ERR_OOM, MRHS_ERR_CUDA = -1, -2, -3, -4
MRHS_ERR_NOCONV, MRHS_ERR_NONFINITE, MRHS_ERR_STATE, MRHS_ERR_TIMEOUT = -5, -6, -7, -8
MRHS_F64, MRHS_F32, MRHS_BF16, MRHS_F16 = 0, 1, 2, 3
MRHS_PREC_FP64, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16 = 0, 1, 2, 3
MRHS_DC_AUTO, MRHS_DC_ALU, MRHS_DC_TC_BF16, MRHS_DC_TC_F16, MRHS_DC_TC_TF32, MRHS_DC_TC_TF32X3 = 0, 1, 2, 3, 4, 5

_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_IP = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes)
_SIGS = {
    "mrhs_create": (_I, [ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _I, _VP, ctypes.POINTER(_VP)]),
    "mrhs_destroy": (None, [_VP]),
    "mrhs_last_error": (ctypes.c_char_p, [_VP]),
    "mrhs_sync": (_I, [_VP]),
    "mrhs_info": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "mrhs_trim": (_I, [_VP]),
    "mrhs_field_bytes": (ctypes.c_size_t, [_VP, _I, _I, _I]),
    "mrhs_get_tables": (_I, [_VP, _VP, _VP, _VP]),
    "mrhs_set_gauge": (_I, [_VP, _VP]),
    "mrhs_build_clover": (_I, [_VP, _D, _D]),
    "mrhs_get_clover": (_I, [_VP, _VP]),
    "mrhs_pack": (_I, [_VP, _VP, _I, _VP, _I, _I]),
    "mrhs_unpack": (_I, [_VP, _VP, _I, _VP, _I, _I]),
    "mrhs_pack_coarse": (_I, [_VP, _VP, _I, _VP, _I, _I]),
    "mrhs_unpack_coarse": (_I, [_VP, _VP, _I, _VP, _I, _I]),
    "mrhs_apply_D": (_I, [_VP, _VP, _VP, _I, _I]),
    "mrhs_apply_D_block": (_I, [_VP, _VP, _VP, _I, _I]),
    "mrhs_sap": (_I, [_VP, _VP, _VP, _I, _I, _I, _I]),
    "mrhs_set_tv": (_I, [_VP, _VP, _I]),
    "mrhs_build_P": (_I, [_VP]),
    "mrhs_build_Dc": (_I, [_VP]),
    "mrhs_set_dc_engine": (_I, [_VP, _I]),
    "mrhs_restrict": (_I, [_VP, _VP, _VP, _I, _I]),
    "mrhs_prolong": (_I, [_VP, _VP, _VP, _I, _I]),
    "mrhs_apply_Dc": (_I, [_VP, _VP, _VP, _I, _I]),
    "mrhs_coarse_solve": (_I, [_VP, _VP, _VP, _I, _I, _D, _I, _I, _VP]),
    "mrhs_coarse_solve_noalloc": (_I, [_VP, _VP, _VP, _I, _I, _D, _I, _I, _VP]),
    "mrhs_setup_init": (_I, [_VP, _VP, _I, _I, _I, _I]),
    "mrhs_setup_refine": (_I, [_VP, _I, _I, _I, _D, _I, _I, _VP]),
    "mrhs_set_block_length": (_I, [_VP, _I]),
    "mrhs_set_smoother": (_I, [_VP, _I]),
    "mrhs_set_coarse_solver": (_I, [_VP, _I]),
    "mrhs_setup_update": (_I, [_VP, _I, _I, _I, _D, _I, _I, _VP]),
    "mrhs_get_tv": (_I, [_VP, _VP, _I]),
    "mrhs_get_P": (_I, [_VP, _VP, _I]),
    "mrhs_get_Dc": (_I, [_VP, _VP, _I]),
    "mrhs_save_setup": (_I, [_VP, ctypes.c_char_p]),
    "mrhs_load_setup": (_I, [_VP, ctypes.c_char_p]),
    "mrhs_profile": (_I, [_VP, _I]),
    "mrhs_profile_read": (_I, [_VP, _I, ctypes.c_char_p, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D)]),
    "mrhs_nn_create": (_I, [_VP, ctypes.POINTER(_I), _I]),
    "mrhs_nn_num_params": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "mrhs_nn_set_weights": (_I, [_VP, _VP]),
    "mrhs_nn_get_weights": (_I, [_VP, _VP, _I]),
    "mrhs_nn_get_grads": (_I, [_VP, _VP]),
    "mrhs_nn_zero_grads": (_I, [_VP]),
    "mrhs_nn_forward": (_I, [_VP, _VP, _VP, _I]),
    "mrhs_nn_infer": (_I, [_VP, _VP, _VP, _I]),
    "mrhs_nn_backward": (_I, [_VP, _VP, _VP, _I]),
    "mrhs_nn_loss": (_I, [_VP, _VP, _VP, _I, _D, ctypes.POINTER(_D), _VP]),
    "mrhs_nn_adam": (_I, [_VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I]),
    "mrhs_nn_train_step": (_I, [_VP, _VP, _I, _D, ctypes.c_float, _I, ctypes.POINTER(_D)]),
    "mrhs_setup_init_learned": (_I, [_VP, _VP, _I, _I, _I]),
    "mrhs_solve_fgmres": (_I, [_VP, _VP, _VP, _D, _I, _I, _D, _I, _I, _I, _I, _VP, _VP]),
}

_lib = None


class MrhsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("mrhs status %d: %s" % (status, msg))
        self.status = status


def lib():
    """Load libmrhs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MrhsError(MRHS_ERR_STATE, "libmrhs.so not built (run paper_1601_03184_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a):
    """Host numpy array or torch tensor (host or device) -> void pointer."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError("cannot pass %r as a pointer" % type(a))


def _nbytes(a):
    """size of a numpy array or torch tensor in bytes (None for a raw pointer)"""
    if isinstance(a, np.ndarray):
        return a.nbytes
    if hasattr(a, "data_ptr"):
        return a.numel() * a.element_size()
    return None


def _fits(ctx, buf, nrhs, dtype, coarse, what):
    """Refuse a numpy array or torch tensor smaller than the field of nrhs
    right-hand sides it is passed as. The library addresses a field by nrhs
    and dtype alone, so a short buffer would be read or written past its end
    on the device. The size needed is the library's own (mrhs_field_bytes);
    raw integer pointers are passed through unchecked."""
    have = _nbytes(buf)
    if have is None:
        return
    need = mrhs_field_bytes(ctx, nrhs, dtype, coarse)
    if have < need:
        raise MrhsError(MRHS_ERR_ARG, "%s: buffer of %d bytes, the %s field of %d right-hand sides needs %d"
                        % (what, have, "coarse" if coarse else "fine", int(nrhs), need))


def _is_torch(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _dev(ctx, buf, nrhs, dtype, coarse, what):
    """A device-field argument: a torch CUDA tensor on the context's GPU (or a
    raw integer device pointer, which the library checks itself). A numpy
    array, a CPU tensor or a tensor on another GPU is refused here, before
    any call, and then held against the field size like _fits."""
    if buf is None or isinstance(buf, int):
        return
    if not _is_torch(buf) or not buf.is_cuda:
        raise MrhsError(MRHS_ERR_ARG, "%s: a device field must be a CUDA tensor, got %s"
                        % (what, "a CPU tensor" if _is_torch(buf) else type(buf).__name__))
    dev = mrhs_info(ctx)[7]
    if buf.device.index is not None and buf.device.index != dev:
        raise MrhsError(MRHS_ERR_ARG, "%s: tensor on cuda:%d, the context lives on cuda:%d"
                        % (what, buf.device.index, dev))
    _fits(ctx, buf, nrhs, dtype, coarse, what)


def _host(buf, what):
    """A host-array argument: numpy or a CPU torch tensor (pinned or not)."""
    if buf is None or isinstance(buf, (int, np.ndarray)):
        return
    if _is_torch(buf) and buf.is_cuda:
        raise MrhsError(MRHS_ERR_ARG, "%s: a host array is required, got a CUDA tensor" % what)


def _check(ctx, st):
    if st != MRHS_OK:
        msg = lib().mrhs_last_error(ctx)
        raise MrhsError(st, msg.decode() if msg else "")
    return st


def _i4(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


# ------------------------------------------------------------ C ABI mirror --
def mrhs_create(dims, agg, ntv, prec, stream=None):
    out = ctypes.c_void_p()
    st = lib().mrhs_create(_i4(dims), _i4(agg), int(ntv), int(prec), stream, ctypes.byref(out))
    _check(None, st)
    return out.value


def mrhs_destroy(ctx):
    lib().mrhs_destroy(ctx)


def mrhs_last_error(ctx):
    m = lib().mrhs_last_error(ctx)
    return m.decode() if m else ""


def mrhs_sync(ctx):
    return _check(ctx, lib().mrhs_sync(ctx))


def mrhs_trim(ctx):
    return _check(ctx, lib().mrhs_trim(ctx))


def mrhs_info(ctx):
    out = (ctypes.c_longlong * 8)()
    _check(ctx, lib().mrhs_info(ctx, out))
    return list(out)


def mrhs_field_bytes(ctx, nrhs, dtype, coarse=0):
    return int(lib().mrhs_field_bytes(ctx, int(nrhs), int(dtype), int(coarse)))


def mrhs_get_tables(ctx, nbr, aggof, aggnbr):
    return _check(ctx, lib().mrhs_get_tables(ctx, _ptr(nbr), _ptr(aggof), _ptr(aggnbr)))


def mrhs_set_gauge(ctx, U):
    return _check(ctx, lib().mrhs_set_gauge(ctx, _ptr(U)))


def mrhs_build_clover(ctx, m0, csw):
    return _check(ctx, lib().mrhs_build_clover(ctx, float(m0), float(csw)))


def mrhs_get_clover(ctx, out):
    return _check(ctx, lib().mrhs_get_clover(ctx, _ptr(out)))


def mrhs_pack(ctx, host, host_dtype, dev, dev_dtype, nrhs):
    _host(host, "mrhs_pack host")
    _dev(ctx, dev, nrhs, dev_dtype, 0, "mrhs_pack")
    return _check(ctx, lib().mrhs_pack(ctx, _ptr(host), host_dtype, _ptr(dev), dev_dtype, int(nrhs)))


def mrhs_unpack(ctx, dev, dev_dtype, host, host_dtype, nrhs):
    _host(host, "mrhs_unpack host")
    _dev(ctx, dev, nrhs, dev_dtype, 0, "mrhs_unpack")
    return _check(ctx, lib().mrhs_unpack(ctx, _ptr(dev), dev_dtype, _ptr(host), host_dtype, int(nrhs)))


def mrhs_pack_coarse(ctx, host, host_dtype, dev, dev_dtype, nrhs):
    _host(host, "mrhs_pack_coarse host")
    _dev(ctx, dev, nrhs, dev_dtype, 1, "mrhs_pack_coarse")
    return _check(ctx, lib().mrhs_pack_coarse(ctx, _ptr(host), host_dtype, _ptr(dev), dev_dtype, int(nrhs)))


def mrhs_unpack_coarse(ctx, dev, dev_dtype, host, host_dtype, nrhs):
    _host(host, "mrhs_unpack_coarse host")
    _dev(ctx, dev, nrhs, dev_dtype, 1, "mrhs_unpack_coarse")
    return _check(ctx, lib().mrhs_unpack_coarse(ctx, _ptr(dev), dev_dtype, _ptr(host), host_dtype, int(nrhs)))


def mrhs_apply_D(ctx, x, y, nrhs, dtype):
    _dev(ctx, x, nrhs, dtype, 0, "mrhs_apply_D x")
    _dev(ctx, y, nrhs, dtype, 0, "mrhs_apply_D y")
    return _check(ctx, lib().mrhs_apply_D(ctx, _ptr(x), _ptr(y), int(nrhs), int(dtype)))


def mrhs_apply_D_block(ctx, x, y, nrhs, dtype):
    _dev(ctx, x, nrhs, dtype, 0, "mrhs_apply_D_block x")
    _dev(ctx, y, nrhs, dtype, 0, "mrhs_apply_D_block y")
    return _check(ctx, lib().mrhs_apply_D_block(ctx, _ptr(x), _ptr(y), int(nrhs), int(dtype)))


def mrhs_sap(ctx, b, x, nrhs, dtype, n_sweeps, n_mr):
    _dev(ctx, b, nrhs, dtype, 0, "mrhs_sap b")
    _dev(ctx, x, nrhs, dtype, 0, "mrhs_sap x")
    return _check(ctx, lib().mrhs_sap(ctx, _ptr(b), _ptr(x), int(nrhs), int(dtype), int(n_sweeps), int(n_mr)))


def mrhs_set_tv(ctx, tv, dtype):
    _dev(ctx, tv, mrhs_info(ctx)[3], dtype, 0, "mrhs_set_tv tv")
    return _check(ctx, lib().mrhs_set_tv(ctx, _ptr(tv), int(dtype)))


def mrhs_build_P(ctx):
    return _check(ctx, lib().mrhs_build_P(ctx))


def mrhs_build_Dc(ctx):
    return _check(ctx, lib().mrhs_build_Dc(ctx))


def mrhs_set_dc_engine(ctx, engine):
    return _check(ctx, lib().mrhs_set_dc_engine(ctx, engine))


def mrhs_restrict(ctx, v, vc, nrhs, dtype):
    _dev(ctx, v, nrhs, dtype, 0, "mrhs_restrict v")
    _dev(ctx, vc, nrhs, dtype, 1, "mrhs_restrict vc")
    return _check(ctx, lib().mrhs_restrict(ctx, _ptr(v), _ptr(vc), int(nrhs), int(dtype)))


def mrhs_prolong(ctx, uc, u, nrhs, dtype):
    _dev(ctx, uc, nrhs, dtype, 1, "mrhs_prolong uc")
    _dev(ctx, u, nrhs, dtype, 0, "mrhs_prolong u")
    return _check(ctx, lib().mrhs_prolong(ctx, _ptr(uc), _ptr(u), int(nrhs), int(dtype)))


def mrhs_apply_Dc(ctx, xc, yc, nrhs, dtype):
    _dev(ctx, xc, nrhs, dtype, 1, "mrhs_apply_Dc xc")
    _dev(ctx, yc, nrhs, dtype, 1, "mrhs_apply_Dc yc")
    return _check(ctx, lib().mrhs_apply_Dc(ctx, _ptr(xc), _ptr(yc), int(nrhs), int(dtype)))


def mrhs_coarse_solve(ctx, bc, xc, nrhs, dtype, tol, restart, maxit):
    _dev(ctx, bc, nrhs, dtype, 1, "mrhs_coarse_solve bc")
    _dev(ctx, xc, nrhs, dtype, 1, "mrhs_coarse_solve xc")
    its = np.zeros(int(nrhs), np.int32)
    _check(ctx, lib().mrhs_coarse_solve(ctx, _ptr(bc), _ptr(xc), int(nrhs), int(dtype), float(tol), int(restart),
                                        int(maxit), _ptr(its)))
    return its


def mrhs_coarse_solve_noalloc(ctx, bc, xc, nrhs, dtype, tol, restart, maxit):
    """mrhs_coarse_solve without allocation (fixed 64 MiB device workspace)."""
    _dev(ctx, bc, nrhs, dtype, 1, "mrhs_coarse_solve_noalloc bc")
    _dev(ctx, xc, nrhs, dtype, 1, "mrhs_coarse_solve_noalloc xc")
    its = np.zeros(int(nrhs), np.int32)
    _check(ctx, lib().mrhs_coarse_solve_noalloc(ctx, _ptr(bc), _ptr(xc), int(nrhs), int(dtype), float(tol),
                                                int(restart), int(maxit), _ptr(its)))
    return its


def mrhs_setup_init(ctx, tv0, dtype, init_mode, n_sweeps, n_mr):
    _dev(ctx, tv0, mrhs_info(ctx)[3], dtype, 0, "mrhs_setup_init tv0")
    return _check(ctx, lib().mrhs_setup_init(ctx, _ptr(tv0), int(dtype), int(init_mode), int(n_sweeps), int(n_mr)))


def mrhs_setup_refine(ctx, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit, ntv=None):
    its = np.zeros((max(int(n_iter), 1), int(ntv or 64)), np.int32)
    _check(ctx, lib().mrhs_setup_refine(ctx, int(n_iter), int(n_sweeps), int(n_mr), float(coarse_tol),
                                        int(coarse_restart), int(coarse_maxit), _ptr(its)))
    return its


def mrhs_setup_update(ctx, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit, ntv=None):
    its = np.zeros((max(int(n_iter), 1), int(ntv or 64)), np.int32)
    _check(ctx, lib().mrhs_setup_update(ctx, int(n_iter), int(n_sweeps), int(n_mr), float(coarse_tol),
                                        int(coarse_restart), int(coarse_maxit), _ptr(its)))
    return its


def mrhs_set_smoother(ctx, even_odd):
    return _check(ctx, lib().mrhs_set_smoother(ctx, int(even_odd)))


def mrhs_set_coarse_solver(ctx, even_odd):
    return _check(ctx, lib().mrhs_set_coarse_solver(ctx, int(even_odd)))


def mrhs_set_block_length(ctx, nb):
    return _check(ctx, lib().mrhs_set_block_length(ctx, int(nb)))


def mrhs_get_tv(ctx, host, host_dtype):
    return _check(ctx, lib().mrhs_get_tv(ctx, _ptr(host), int(host_dtype)))


def mrhs_get_P(ctx, host, host_dtype):
    return _check(ctx, lib().mrhs_get_P(ctx, _ptr(host), int(host_dtype)))


def mrhs_get_Dc(ctx, host, host_dtype):
    return _check(ctx, lib().mrhs_get_Dc(ctx, _ptr(host), int(host_dtype)))


def mrhs_save_setup(ctx, path):
    return _check(ctx, lib().mrhs_save_setup(ctx, os.fsencode(str(path))))


def mrhs_load_setup(ctx, path):
    return _check(ctx, lib().mrhs_load_setup(ctx, os.fsencode(str(path))))


def mrhs_profile(ctx, enable):
    return _check(ctx, lib().mrhs_profile(ctx, int(enable)))


def mrhs_profile_read(ctx):
    """All per-kernel totals: {name: (launches, total_ms)}."""
    out = {}
    i = 0
    name = ctypes.create_string_buffer(64)
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0)
    while lib().mrhs_profile_read(ctx, i, name, 64, ctypes.byref(n), ctypes.byref(ms)) == MRHS_OK:
        out[name.value.decode()] = (n.value, ms.value)
        i += 1
    return out


def mrhs_nn_create(ctx, widths, bf16_weights=1):
    return _check(ctx, lib().mrhs_nn_create(ctx, _i4(widths), int(bf16_weights)))


def mrhs_nn_num_params(ctx):
    a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(ctx, lib().mrhs_nn_num_params(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mrhs_nn_set_weights(ctx, host):
    return _check(ctx, lib().mrhs_nn_set_weights(ctx, _ptr(np.ascontiguousarray(host, dtype=np.float32))))


def mrhs_nn_get_weights(ctx, compute_copy=0):
    nc, nr = mrhs_nn_num_params(ctx)
    out = np.zeros(2 * nc + nr, np.float32)
    _check(ctx, lib().mrhs_nn_get_weights(ctx, _ptr(out), int(compute_copy)))
    return out


def mrhs_nn_get_grads(ctx):
    nc, nr = mrhs_nn_num_params(ctx)
    out = np.zeros(2 * nc + nr, np.float32)
    _check(ctx, lib().mrhs_nn_get_grads(ctx, _ptr(out)))
    return out


def mrhs_nn_zero_grads(ctx):
    return _check(ctx, lib().mrhs_nn_zero_grads(ctx))


def mrhs_nn_forward(ctx, x, y, nrhs):
    _dev(ctx, x, nrhs, MRHS_F32, 0, "mrhs_nn_forward in")
    _dev(ctx, y, nrhs, MRHS_F32, 0, "mrhs_nn_forward out")
    return _check(ctx, lib().mrhs_nn_forward(ctx, _ptr(x), _ptr(y), int(nrhs)))


def mrhs_nn_infer(ctx, x, y, nrhs):
    _dev(ctx, x, nrhs, MRHS_F32, 0, "mrhs_nn_infer in")
    _dev(ctx, y, nrhs, MRHS_F32, 0, "mrhs_nn_infer out")
    return _check(ctx, lib().mrhs_nn_infer(ctx, _ptr(x), _ptr(y), int(nrhs)))


def mrhs_nn_backward(ctx, gout, gin, nrhs):
    _dev(ctx, gout, nrhs, MRHS_F32, 0, "mrhs_nn_backward grad_out")
    _dev(ctx, gin, nrhs, MRHS_F32, 0, "mrhs_nn_backward grad_in")
    return _check(ctx, lib().mrhs_nn_backward(ctx, _ptr(gout), _ptr(gin), int(nrhs)))


def mrhs_nn_loss(ctx, v, gv, nrhs, lam):
    _dev(ctx, v, nrhs, MRHS_F32, 0, "mrhs_nn_loss v")
    _dev(ctx, gv, nrhs, MRHS_F32, 0, "mrhs_nn_loss grad_v")
    loss = ctypes.c_double(0)
    per = np.zeros(int(nrhs), np.float64)
    _check(ctx, lib().mrhs_nn_loss(ctx, _ptr(v), _ptr(gv), int(nrhs), float(lam), ctypes.byref(loss), _ptr(per)))
    return loss.value, per


def mrhs_nn_adam(ctx, lr, beta1, beta2, eps, step):
    return _check(ctx, lib().mrhs_nn_adam(ctx, float(lr), float(beta1), float(beta2), float(eps), int(step)))


def mrhs_nn_train_step(ctx, v_in, nrhs, lam, lr, step):
    _dev(ctx, v_in, nrhs, MRHS_F32, 0, "mrhs_nn_train_step v_in")
    loss = ctypes.c_double(0)
    _check(ctx, lib().mrhs_nn_train_step(ctx, _ptr(v_in), int(nrhs), float(lam), float(lr), int(step),
                                         ctypes.byref(loss)))
    return loss.value


def mrhs_setup_init_learned(ctx, tv0, dtype, n_sweeps, n_mr):
    _dev(ctx, tv0, mrhs_info(ctx)[3], dtype, 0, "mrhs_setup_init_learned tv0")
    return _check(ctx, lib().mrhs_setup_init_learned(ctx, _ptr(tv0), int(dtype), int(n_sweeps), int(n_mr)))


def mrhs_solve_fgmres(ctx, b, x, tol, restart, maxit, coarse_tol, coarse_restart, coarse_maxit, n_sweeps, n_mr,
                      allow_noconv=False):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = lib().mrhs_solve_fgmres(ctx, _ptr(b), _ptr(x), float(tol), int(restart), int(maxit), float(coarse_tol),
                                 int(coarse_restart), int(coarse_maxit), int(n_sweeps), int(n_mr),
                                 ctypes.addressof(it), ctypes.addressof(rr))
    if not (allow_noconv and st == MRHS_ERR_NOCONV):
        _check(ctx, st)
    return it.value, rr.value, st


from .lattice import Lattice  # noqa: E402  (convenience wrapper over the functions above)
