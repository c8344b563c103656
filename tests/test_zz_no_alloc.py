"""The allocation-free coarse solve (mrhs_coarse_solve_noalloc) against the
ordinary one (mrhs_coarse_solve), through the C ABI on the GPU.

Callers whose device memory is owned entirely by their own allocator, or who
must not trigger the device-wide synchronisation of cudaMalloc in the middle
of a solve, use the allocation-free entry point; it keeps its workspace in a
fixed device array inside the library, shared by all calls. This file is
collected last so that a failure here cannot stop the other tests."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_SHAPE, MRHS_F32, MRHS_F64, MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice,
                                    MrhsError,
                                    mrhs_coarse_solve, mrhs_coarse_solve_noalloc, inputs)

pytestmark = pytest.mark.gpu

DIMS, AGG, NTV = (4, 4, 4, 4), (2, 2, 2, 2), 8


@pytest.fixture(scope="module")
def lat():
    U = inputs.gauge_field(DIMS, 0.3, 1001)
    lat = Lattice(DIMS, AGG, NTV, MRHS_PREC_FP64)
    lat.set_gauge(U)
    lat.build_clover(-0.2, 1.0)
    lat.set_tv(lat.to_device(inputs.test_vectors(NTV, DIMS, 2001), MRHS_F64), MRHS_F64)
    lat.build_P()
    lat.build_Dc()
    return lat


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_coarse_solve_on_two_calls_in_a_row(lat):
    nrhs = 4
    for call, seed in enumerate((4001, 4002)):
        bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * NTV), seed)
        if call == 1:
            bc[1] = 0  # a zero right-hand side: x stays 0 and no iteration is done
        bcd = lat.to_device(bc, MRHS_F64, coarse=True)
        ref = lat.field(nrhs, MRHS_F64, coarse=True)
        got = lat.field(nrhs, MRHS_F64, coarse=True)
        got.fill_(255)  # stale contents must not matter
        its_ref = mrhs_coarse_solve(lat.ctx, bcd, ref, nrhs, MRHS_F64, 1e-8, 10, 200)
        its = mrhs_coarse_solve_noalloc(lat.ctx, bcd, got, nrhs, MRHS_F64, 1e-8, 10, 200)
        assert list(its) == list(its_ref)
        x_ref = lat.to_host(ref, nrhs, MRHS_F64, coarse=True)
        x = lat.to_host(got, nrhs, MRHS_F64, coarse=True)
        assert _rel(x, x_ref) < 1e-12
        # and it is a solution: |b - Dc x| <= 1e-8 |b| for every non-zero right-hand side
        res = bc - oracle.apply_Dc(DIMS, AGG, lat.get_Dc(), x)
        for r in range(nrhs):
            if np.linalg.norm(bc[r]) > 0:
                assert np.linalg.norm(res[r]) <= 1.0001e-8 * np.linalg.norm(bc[r])
            else:
                assert np.abs(x[r]).max() == 0


def test_noalloc_rejects_problems_beyond_its_workspace(lat):
    nrhs = 256  # (restart + 2) * 256 right-hand sides of 256 coarse rows > 64 MiB
    bcd = lat.field(nrhs, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    with pytest.raises(MrhsError) as e:
        mrhs_coarse_solve_noalloc(lat.ctx, bcd, xcd, nrhs, MRHS_F64, 0.05, 64, 10)
    assert e.value.status == MRHS_ERR_SHAPE
    assert "64" in str(e.value) or "bytes" in str(e.value)


def test_noalloc_fp32_tensor_core_path_is_bit_identical():
    """FP32 context with 16 right-hand sides and 2 N_tv = 16: the coarse
    stencil inside both solves runs on the tensor cores, and the four-wide
    reductions and updates read the Krylov basis from the library's fixed
    array (16-byte aligned rows). The two entry points run the same kernels
    on the same data, so iteration counts and x agree bit for bit."""
    dims, agg, ntv, nrhs = (8, 8, 8, 8), (4, 4, 4, 4), 8, 16
    U = inputs.gauge_field(dims, 0.4, 1301)
    lat32 = Lattice(dims, agg, ntv, MRHS_PREC_FP32)
    lat32.set_gauge(U)
    lat32.build_clover(-0.1, 1.2)
    lat32.set_tv(lat32.to_device(inputs.test_vectors(ntv, dims, 2301).astype(np.complex64), MRHS_F32), MRHS_F32)
    lat32.build_P()
    lat32.build_Dc()
    for seed in (4101, 4102):
        bc = inputs.gaussian_field((nrhs, lat32.nagg, 2 * ntv), seed).astype(np.complex64)
        bcd = lat32.to_device(bc, MRHS_F32, coarse=True)
        ref = lat32.field(nrhs, MRHS_F32, coarse=True)
        got = lat32.field(nrhs, MRHS_F32, coarse=True)
        got.fill_(255)
        its_ref = mrhs_coarse_solve(lat32.ctx, bcd, ref, nrhs, MRHS_F32, 1e-5, 8, 60)
        its = mrhs_coarse_solve_noalloc(lat32.ctx, bcd, got, nrhs, MRHS_F32, 1e-5, 8, 60)
        assert list(its) == list(its_ref)
        assert bool((ref == got).all())
    lat32.close()
