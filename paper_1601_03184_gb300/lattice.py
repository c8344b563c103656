"""Convenience wrapper: one lattice context plus torch-allocated device fields.

Only argument marshalling: device memory comes from torch (the caching
allocator), every operation is one call of the C ABI.
"""
from __future__ import annotations

import numpy as np

from . import (MRHS_F32, MRHS_F64, MRHS_PREC_FP64, mrhs_apply_D, mrhs_apply_D_block, mrhs_apply_Dc,
               mrhs_build_clover, mrhs_build_Dc, mrhs_build_P, mrhs_coarse_solve, mrhs_create, mrhs_destroy,
               mrhs_set_dc_engine,
               mrhs_field_bytes, mrhs_get_clover, mrhs_get_Dc, mrhs_get_P, mrhs_get_tables, mrhs_get_tv,
               mrhs_info, mrhs_load_setup, mrhs_pack, mrhs_pack_coarse, mrhs_prolong, mrhs_restrict, mrhs_sap,
               mrhs_save_setup, mrhs_set_block_length, mrhs_set_coarse_solver, mrhs_set_gauge,
               mrhs_set_smoother,
               mrhs_setup_update,
               mrhs_set_tv, mrhs_setup_init, mrhs_setup_refine, mrhs_solve_fgmres, mrhs_sync, mrhs_unpack,
               mrhs_unpack_coarse)

_HOST_NP = {MRHS_F64: np.complex128, MRHS_F32: np.complex64}


class Lattice:
    def __init__(self, dims, agg, ntv, prec=MRHS_PREC_FP64, stream=None):
        import torch

        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.agg = tuple(int(a) for a in agg)
        self.ntv = int(ntv)
        self.prec = int(prec)
        self.V = int(np.prod(self.dims))
        self.nagg = int(np.prod([d // a for d, a in zip(self.dims, self.agg)]))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.ctx = mrhs_create(self.dims, self.agg, self.ntv, self.prec, stream)

    def close(self):
        if self.ctx:
            mrhs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ fields --
    def field(self, nrhs, dtype, coarse=False, zero=True):
        n = mrhs_field_bytes(self.ctx, nrhs, dtype, 1 if coarse else 0)
        t = self.torch.empty(n, dtype=self.torch.uint8, device="cuda")
        if zero:
            t.zero_()
        return t

    def to_device(self, host, dtype, coarse=False):
        """host [nrhs, V, 12] (or [nrhs, nagg, 2ntv] for coarse) complex -> device field"""
        hd = MRHS_F64 if host.dtype == np.complex128 else MRHS_F32
        host = np.ascontiguousarray(host, dtype=np.complex128 if hd == MRHS_F64 else np.complex64)
        want = (self.nagg, 2 * self.ntv) if coarse else (self.V, 12)
        if host.ndim != 3 or host.shape[1:] != want:
            raise ValueError("host field must be [nrhs, %d, %d], got %s" % (want + (host.shape,)))
        nrhs = host.shape[0]
        d = self.field(nrhs, dtype, coarse, zero=False)
        (mrhs_pack_coarse if coarse else mrhs_pack)(self.ctx, host, hd, d, dtype, nrhs)
        return d

    def to_host(self, dev, nrhs, dtype, coarse=False, host_dtype=MRHS_F64):
        shape = (nrhs, self.nagg, 2 * self.ntv) if coarse else (nrhs, self.V, 12)
        out = np.empty(shape, _HOST_NP[host_dtype])
        (mrhs_unpack_coarse if coarse else mrhs_unpack)(self.ctx, dev, dtype, out, host_dtype, nrhs)
        return out

    # ------------------------------------------------------------- setup --
    def set_gauge(self, U):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        if U.size != self.V * 36:
            raise ValueError("gauge field must hold [V, 4, 3, 3] = %d complex numbers, got %d" % (self.V * 36, U.size))
        mrhs_set_gauge(self.ctx, U)

    def build_clover(self, m0, csw):
        mrhs_build_clover(self.ctx, m0, csw)

    def clover(self):
        out = np.empty((self.V, 2, 6, 6), np.complex128)
        mrhs_get_clover(self.ctx, out)
        return out

    def tables(self):
        nbr = np.empty((self.V, 8), np.int32)
        aggof = np.empty((self.V, 2), np.int32)
        aggnbr = np.empty((self.nagg, 8), np.int32)
        mrhs_get_tables(self.ctx, nbr, aggof, aggnbr)
        return nbr, aggof, aggnbr

    def apply_D(self, x, y, nrhs, dtype):
        mrhs_apply_D(self.ctx, x, y, nrhs, dtype)

    def apply_D_block(self, x, y, nrhs, dtype):
        mrhs_apply_D_block(self.ctx, x, y, nrhs, dtype)

    def sap(self, b, x, nrhs, dtype, n_sweeps, n_mr):
        mrhs_sap(self.ctx, b, x, nrhs, dtype, n_sweeps, n_mr)

    def set_tv(self, tv, dtype):
        mrhs_set_tv(self.ctx, tv, dtype)

    def build_P(self):
        mrhs_build_P(self.ctx)

    def build_Dc(self):
        mrhs_build_Dc(self.ctx)

    def set_dc_engine(self, engine):
        mrhs_set_dc_engine(self.ctx, engine)

    def restrict(self, v, vc, nrhs, dtype):
        mrhs_restrict(self.ctx, v, vc, nrhs, dtype)

    def prolong(self, uc, u, nrhs, dtype):
        mrhs_prolong(self.ctx, uc, u, nrhs, dtype)

    def apply_Dc(self, xc, yc, nrhs, dtype):
        mrhs_apply_Dc(self.ctx, xc, yc, nrhs, dtype)

    def coarse_solve(self, bc, xc, nrhs, dtype, tol, restart, maxit):
        return mrhs_coarse_solve(self.ctx, bc, xc, nrhs, dtype, tol, restart, maxit)

    def setup_init(self, tv0, dtype, init_mode=0, n_sweeps=3, n_mr=4):
        mrhs_setup_init(self.ctx, tv0, dtype, init_mode, n_sweeps, n_mr)

    def setup_update(self, n_iter, n_sweeps=4, n_mr=4, coarse_tol=0.05, coarse_restart=20, coarse_maxit=200):
        """after set_gauge + build_clover of a changed field: D_c from the kept P,
        then n_iter refinement iterations from the kept test vectors"""
        its = mrhs_setup_update(self.ctx, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit,
                                ntv=self.ntv)
        return its[:n_iter]

    def set_smoother(self, even_odd):
        """1: even-odd preconditioned SAP domain solves, 0: plain"""
        mrhs_set_smoother(self.ctx, even_odd)

    def set_coarse_solver(self, even_odd):
        """1: coarse GMRES on the Schur complement of the even aggregates, 0: on D_c"""
        mrhs_set_coarse_solver(self.ctx, even_odd)

    def set_block_length(self, nb):
        """N_b of Algorithm 2 for the setup phases (0: all test vectors at once)"""
        mrhs_set_block_length(self.ctx, nb)

    def setup_refine(self, n_iter, n_sweeps=4, n_mr=4, coarse_tol=0.05, coarse_restart=20, coarse_maxit=200):
        its = mrhs_setup_refine(self.ctx, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit,
                                ntv=self.ntv)
        return its[:n_iter]

    def get_tv(self, host_dtype=MRHS_F64):
        out = np.empty((self.ntv, self.V, 12), _HOST_NP[host_dtype])
        mrhs_get_tv(self.ctx, out, host_dtype)
        return out

    def get_P(self, host_dtype=MRHS_F64):
        out = np.empty((self.ntv, self.V, 12), _HOST_NP[host_dtype])
        mrhs_get_P(self.ctx, out, host_dtype)
        return out

    def get_Dc(self, host_dtype=MRHS_F64):
        nc = 2 * self.ntv
        out = np.empty((self.nagg, 9, nc, nc), _HOST_NP[host_dtype])
        mrhs_get_Dc(self.ctx, out, host_dtype)
        return out

    def solve_fgmres(self, b, tol=1e-10, restart=25, maxit=500, coarse_tol=0.05, coarse_restart=20,
                     coarse_maxit=200, n_sweeps=4, n_mr=4, allow_noconv=False):
        b = np.ascontiguousarray(b, dtype=np.complex128).reshape(self.V, 12)
        x = np.zeros_like(b)
        it, rr, st = mrhs_solve_fgmres(self.ctx, b, x, tol, restart, maxit, coarse_tol, coarse_restart,
                                       coarse_maxit, n_sweeps, n_mr, allow_noconv=allow_noconv)
        return x, it, rr

    def save_setup(self, path):
        mrhs_save_setup(self.ctx, path)

    def load_setup(self, path):
        mrhs_load_setup(self.ctx, path)

    def info(self):
        return mrhs_info(self.ctx)

    def sync(self):
        mrhs_sync(self.ctx)
