"""Tensor-core (tcgen05) contraction of the coarse operator D_c = P^dag D P
against the FP64 oracle evaluated on the same P.

The tensor-core path computes C = P^dag Y with Y = D_k P (FP32 on the CUDA
cores) rounded to the operand type (unit roundoff u: bf16 2^-8, fp16 and tf32
2^-11, split tf32 2^-21 for the sum of the three partial products), P rounded
to it as well (exact when P is stored in bf16 / fp16), and
FP32 accumulation over the K = 2 * 12 * |block| real products. Each entry
therefore obeys
  |C_gpu[i][j] - C[i][j]| <= (2u + K 2^-24 + e_Y) sum_n |P_ni| |Y_nj|
                           <= (2u + K 2^-24 + e_Y) ||P_i|| ||Y_j||,
e_Y = 1e-5 the FP32 error of Y itself. ||Y_j|| is the norm of D_B P_j on the
aggregate for the self block (D_B: D without couplings between aggregates,
from the oracle) and at most ||P_j|| on the neighbouring aggregate for a
hopping block (one hop is a projector times a unitary link). The test asserts
this bound with a factor 2, entry by entry, on every block including the
backward blocks derived by gamma_5-hermiticity; the CUDA-core engine on the
same P stays at FP32 accuracy.
"""
import numpy as np
import pytest

import oracle
from lattice_helpers import aggregate_of_sites
from paper_1601_03184_gb300 import (MRHS_DC_ALU, MRHS_DC_AUTO, MRHS_DC_TC_BF16, MRHS_DC_TC_F16, MRHS_DC_TC_TF32,
                                    MRHS_DC_TC_TF32X3,
                                    MRHS_ERR_SHAPE, MRHS_F32, MRHS_PREC_FP32, MRHS_PREC_FP64, MRHS_PREC_MIX_BF16,
                                    MRHS_PREC_MIX_FP16, Lattice, MrhsError, inputs)

pytestmark = pytest.mark.gpu

CASES = {
    # the paper's 4^4 aggregates with N_tv = 32: M = 128 rows, N = 128 columns, full chunks
    "4^4-ntv32": dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=32, eps=0.5, m0=-0.3, csw=1.5, gseed=1401, tvseed=2401),
    # ragged aggregates (face sizes 12 and 8: partial chunks), 2*2ntv = 24 padded to N = 32
    "ragged-ntv6": dict(dims=(4, 6, 4, 8), agg=(2, 3, 2, 2), ntv=6, eps=0.5, m0=0.1, csw=1.3, gseed=1101, tvseed=2402),
    # 2^4 aggregates, N_tv = 8
    "2^4-ntv8": dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2403),
}
# (context precision, engine, unit roundoff of the operands)
ENGINES = {
    "mixbf16-auto": (MRHS_PREC_MIX_BF16, MRHS_DC_AUTO, 2.0 ** -8),
    "mixfp16-auto": (MRHS_PREC_MIX_FP16, MRHS_DC_AUTO, 2.0 ** -11),
    "fp32-bf16": (MRHS_PREC_FP32, MRHS_DC_TC_BF16, 2.0 ** -8),
    "fp32-f16": (MRHS_PREC_FP32, MRHS_DC_TC_F16, 2.0 ** -11),
    "fp32-tf32": (MRHS_PREC_FP32, MRHS_DC_TC_TF32, 2.0 ** -11),
    # split tf32 (hi + lo parts): each operand to 2^-22, the dropped lo*lo term below 2^-22
    "fp32-tf32x3": (MRHS_PREC_FP32, MRHS_DC_TC_TF32X3, 2.0 ** -21),
}


def setup_P(cfg, prec, engine):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    lat.set_dc_engine(engine)
    tv = inputs.test_vectors(cfg["ntv"], cfg["dims"], cfg["tvseed"]).astype(np.complex64)
    lat.set_tv(lat.to_device(tv, MRHS_F32), MRHS_F32)
    lat.build_P()
    return lat, U, A


def column_fields(P):
    """[2 ntv, V, 12]: column (h, j) = P_j restricted to chirality h"""
    ntv = P.shape[0]
    cols = np.zeros((2 * ntv,) + P.shape[1:], P.dtype)
    for h in range(2):
        cols[h * ntv:(h + 1) * ntv, :, 6 * h:6 * h + 6] = P[:, :, 6 * h:6 * h + 6]
    return cols


def entry_bounds(cfg, U, A, P, gamma):
    """tolerance per entry of D_c [nagg, 9, nc, nc] from the bound above"""
    dims, agg = cfg["dims"], cfg["agg"]
    Ag = aggregate_of_sites(dims, agg)
    nagg = int(Ag.max()) + 1
    cols = column_fields(P)
    Y = oracle.apply_D_block(dims, agg, U, A, cols)
    pn = np.zeros((nagg, cols.shape[0]))
    yn = np.zeros((nagg, cols.shape[0]))
    for a in range(nagg):
        m = Ag == a
        pn[a] = np.sqrt((np.abs(cols[:, m, :]) ** 2).sum(axis=(1, 2)))
        yn[a] = np.sqrt((np.abs(Y[:, m, :]) ** 2).sum(axis=(1, 2)))
    nc = cols.shape[0]
    tol = np.empty((nagg, 9, nc, nc))
    pmax = pn.max()
    for a in range(nagg):
        tol[a, 0] = gamma * np.outer(pn[a], yn[a])
        tol[a, 1:] = gamma * pmax * pmax
    return tol


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("eng", list(ENGINES))
def test_coarse_op_tensor_cores(case, eng):
    cfg = CASES[case]
    prec, engine, u = ENGINES[eng]
    lat, U, A = setup_P(cfg, prec, engine)
    lat.build_Dc()
    P = lat.get_P()
    Dc = lat.get_Dc()
    Dref = oracle.coarse_op(cfg["dims"], cfg["agg"], U, A, P)
    Va = int(np.prod(cfg["agg"]))
    gamma = 2.0 * (2 * u + 24 * Va * 2.0 ** -24 + 1e-5)
    tol = entry_bounds(cfg, U, A, P, gamma)
    err = np.abs(Dc - Dref)
    worst = (err / tol).max()
    print("%s %s: max |dDc| %.3e, max |dDc|/bound %.3f, rel %.3e" %
          (case, eng, err.max(), worst, np.linalg.norm(Dc - Dref) / np.linalg.norm(Dref)))
    assert worst <= 1.0
    # the same P through the CUDA-core contraction: FP32 accuracy
    lat.set_dc_engine(MRHS_DC_ALU)
    lat.build_Dc()
    assert np.linalg.norm(lat.get_Dc() - Dref) / np.linalg.norm(Dref) < 1e-5


def test_tensor_core_engine_is_used_and_differs_from_alu():
    """the tensor-core result carries the operand rounding (so the kernel ran),
    and is bitwise reproducible"""
    cfg = CASES["4^4-ntv32"]
    lat, U, A = setup_P(cfg, MRHS_PREC_FP32, MRHS_DC_TC_BF16)
    lat.build_Dc()
    d1 = lat.get_Dc()
    lat.build_Dc()
    assert np.array_equal(d1, lat.get_Dc())
    lat.set_dc_engine(MRHS_DC_ALU)
    lat.build_Dc()
    d2 = lat.get_Dc()
    r = np.linalg.norm(d1 - d2) / np.linalg.norm(d2)
    assert 1e-5 < r < 2.0 ** -7


def test_engine_argument_checks():
    cfg = CASES["2^4-ntv8"]
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], MRHS_PREC_FP64)
    with pytest.raises(MrhsError):
        lat.set_dc_engine(7)
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    tv = inputs.test_vectors(cfg["ntv"], cfg["dims"], cfg["tvseed"])
    from paper_1601_03184_gb300 import MRHS_F64
    lat.set_tv(lat.to_device(tv, MRHS_F64), MRHS_F64)
    lat.build_P()
    lat.set_dc_engine(MRHS_DC_TC_BF16)  # FP64 work fields: no tensor-core form
    with pytest.raises(MrhsError) as e:
        lat.build_Dc()
    assert e.value.status == MRHS_ERR_SHAPE


@pytest.mark.parametrize("prec", [MRHS_PREC_FP32, MRHS_PREC_MIX_BF16], ids=["fp32-split", "bf16-tf32"])
@pytest.mark.parametrize("nrhs", [16, 32])
def test_apply_Dc_tensor_cores(prec, nrhs):
    """y_c = D_c x_c on the tensor cores against the oracle's stencil on the
    same D_c and x_c. Per entry |dy_ir| <= gamma sum_k sum_j |D[A,k]_ij| |x_jr|
    with gamma = 2 (2 e + K 2^-24), K = 2 * 9 * 2 N_tv real products per
    output and e the operand error: 2^-22 per part for split tf32 (v = hi + lo
    to 22 bits, the dropped lo*lo below 2^-22), 2^-11 for single tf32."""
    cfg = CASES["4^4-ntv32"]
    lat, U, A = setup_P(cfg, prec, MRHS_DC_AUTO)
    lat.build_Dc()
    Dc = lat.get_Dc()
    nc = 2 * cfg["ntv"]
    xc = inputs.gaussian_field((nrhs, lat.nagg, nc), 901).astype(np.complex64)
    xd = lat.to_device(xc, MRHS_F32, coarse=True)
    yd = lat.field(nrhs, MRHS_F32, coarse=True)
    lat.apply_Dc(xd, yd, nrhs, MRHS_F32)
    lat.sync()
    y = lat.to_host(yd, nrhs, MRHS_F32, coarse=True)
    x64 = xc.astype(np.complex128)
    yref = oracle.apply_Dc(cfg["dims"], cfg["agg"], Dc, x64)
    _, _, aggnbr = lat.tables()
    S = np.zeros(yref.shape)
    absD, absx = np.abs(Dc), np.abs(x64)
    for k in range(9):
        B = np.arange(lat.nagg) if k == 0 else aggnbr[:, k - 1]
        S += np.einsum("aij,raj->rai", absD[:, k], absx[:, B, :])
    e = 2.0 ** -22 if prec == MRHS_PREC_FP32 else 2.0 ** -11
    gamma = 2.0 * (2 * e + 2 * 9 * nc * 2.0 ** -24)
    worst = (np.abs(y - yref) / (gamma * S)).max()
    print("apply_Dc prec %d nrhs %d: rel %.3e, max |dy|/bound %.3f" % (prec, nrhs, rel_err(y, yref), worst))
    assert worst <= 1.0
    if prec == MRHS_PREC_FP32:
        # the split really carries the low parts: one tf32 rounding of the
        # operands alone would leave a relative error near 2^-12
        assert rel_err(y, yref) < 2.0 ** -11 / 16


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _apply_Dc_result(prec, nrhs):
    cfg = CASES["4^4-ntv32"]
    lat, _, _ = setup_P(cfg, prec, MRHS_DC_AUTO)
    lat.build_Dc()
    xc = inputs.gaussian_field((nrhs, lat.nagg, 2 * cfg["ntv"]), 902).astype(np.complex64)
    yd = lat.field(nrhs, MRHS_F32, coarse=True)
    lat.apply_Dc(lat.to_device(xc, MRHS_F32, coarse=True), yd, nrhs, MRHS_F32)
    lat.sync()
    return lat.to_host(yd, nrhs, MRHS_F32, coarse=True, host_dtype=MRHS_F32)


@pytest.mark.parametrize("prec", [MRHS_PREC_FP32, MRHS_PREC_MIX_BF16], ids=["fp32-split", "bf16-tf32"])
def test_apply_Dc_images_equal_block_conversion(prec, tmp_path):
    """The coarse stencil reads D_c as the operand images made when D_c is
    built; with MRHS_DC_IMAGES=0 (a child process, the switch is read once) it
    converts every block itself. Both hold the same tf32 parts in the same
    layout and run the same MMAs, so the results are equal bit for bit."""
    import os
    import subprocess
    import sys
    nrhs = 32
    y_img = _apply_Dc_result(prec, nrhs)
    out = tmp_path / "y.npy"
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); import numpy as np; "
            "import test_gpu_tc as t; np.save(%r, t._apply_Dc_result(%d, %d))"
            % (here, os.path.dirname(here), str(out), prec, nrhs))
    env = dict(os.environ, MRHS_DC_IMAGES="0")
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=os.path.dirname(here), timeout=600)
    y_conv = np.load(out)
    assert y_img.dtype == y_conv.dtype and np.array_equal(y_img.view(np.uint32), y_conv.view(np.uint32))
