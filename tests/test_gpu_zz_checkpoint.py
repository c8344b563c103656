"""Checkpoint and restore of a finished setup (mrhs_save_setup /
mrhs_load_setup) through the C ABI on the GPU, with N_tv = 8 in all four
precisions: FP64 on a 4^4 lattice with 2^4 domains, the reduced precisions on
an 8^4 lattice with 4^4 domains.

A restored setup must equal the saved one bit for bit (test vectors, P, D_c)
and must act the same: the coarse stencil gives identical results, the
two-level FGMRES solve converges as with the original, and (FP64, whose setup
is deterministic) a further refinement iteration from the restored setup
gives the same P and D_c as one from the original. Files from another
geometry, damaged or truncated files, and a save before the setup are
refused with the documented status codes.
"""
import os

import numpy as np
import pytest

from paper_1601_03184_gb300 import (MRHS_ERR_ARG, MRHS_ERR_SHAPE, MRHS_ERR_STATE, MRHS_F32, MRHS_F64,
                                    MRHS_PREC_FP32, MRHS_PREC_FP64, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16,
                                    Lattice, MrhsError, inputs, mrhs_load_setup, mrhs_save_setup)

pytestmark = pytest.mark.gpu

SMALL = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)
LARGE = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1201, tvseed=2201)
PRECS = [MRHS_PREC_FP64, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16]
IDS = ["fp64", "fp32", "bf16", "fp16"]


def config(prec):
    return SMALL if prec == MRHS_PREC_FP64 else LARGE


def make(prec, ntv=None):
    cfg = config(prec)
    lat = Lattice(cfg["dims"], cfg["agg"], ntv or cfg["ntv"], prec)
    lat.set_gauge(inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"]))
    lat.build_clover(cfg["m0"], cfg["csw"])
    return lat


def run_setup(lat, prec):
    tv0 = inputs.test_vectors(lat.ntv, lat.dims, config(prec)["tvseed"])
    if prec == MRHS_PREC_FP64:
        lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 3, 4)
    else:
        lat.setup_init(lat.to_device(tv0.astype(np.complex64), MRHS_F32), MRHS_F32, 0, 3, 4)
    lat.setup_refine(1, 4, 4, 0.05, 20, 200)


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
def test_restored_setup_is_the_saved_one(tmp_path, prec):
    path = str(tmp_path / "setup.bin")
    src = make(prec)
    run_setup(src, prec)
    mrhs_save_setup(src.ctx, path)
    assert os.path.exists(path) and not os.path.exists(path + ".part")
    dst = make(prec)
    mrhs_load_setup(dst.ctx, path)
    assert np.array_equal(dst.get_tv(), src.get_tv())
    assert np.array_equal(dst.get_P(), src.get_P())
    assert np.array_equal(dst.get_Dc(), src.get_Dc())

    # the coarse stencil on the restored D_c
    wd = MRHS_F64 if prec == MRHS_PREC_FP64 else MRHS_F32
    nrhs = 4
    xc = inputs.gaussian_field((nrhs, src.nagg, 2 * src.ntv), 4301)
    ys = []
    for lat in (src, dst):
        y = lat.field(nrhs, wd, coarse=True)
        lat.apply_Dc(lat.to_device(xc, wd, coarse=True), y, nrhs, wd)
        ys.append(lat.to_host(y, nrhs, wd, coarse=True))
    assert np.array_equal(ys[0], ys[1])

    # the two-level solve with the restored setup
    b = inputs.gaussian_field((src.V, 12), 4302)
    _, its_src, _ = src.solve_fgmres(b, tol=1e-10, restart=25, maxit=400)
    _, its_dst, rr = dst.solve_fgmres(b, tol=1e-10, restart=25, maxit=400)
    assert rr <= 1e-10
    assert abs(its_dst - its_src) <= 1

    if prec == MRHS_PREC_FP64:
        # refinement continues from the restored setup exactly as from the original
        for lat in (src, dst):
            lat.setup_refine(1, 4, 4, 0.05, 20, 200)
        assert np.array_equal(dst.get_P(), src.get_P())
        assert np.array_equal(dst.get_Dc(), src.get_Dc())
    src.close()
    dst.close()


def test_checkpoint_errors(tmp_path):
    prec = MRHS_PREC_FP64
    path = str(tmp_path / "setup.bin")
    fresh = make(prec)
    with pytest.raises(MrhsError) as e:
        mrhs_save_setup(fresh.ctx, path)
    assert e.value.status == MRHS_ERR_STATE
    assert not os.path.exists(path) and not os.path.exists(path + ".part")
    with pytest.raises(MrhsError) as e:
        mrhs_load_setup(fresh.ctx, str(tmp_path / "missing.bin"))
    assert e.value.status == MRHS_ERR_ARG

    src = make(prec)
    run_setup(src, prec)
    mrhs_save_setup(src.ctx, path)
    data = open(path, "rb").read()

    # another N_tv: refused before anything is read into the context
    other = make(prec, ntv=4)
    with pytest.raises(MrhsError) as e:
        mrhs_load_setup(other.ctx, path)
    assert e.value.status == MRHS_ERR_SHAPE

    # not a checkpoint
    junk = str(tmp_path / "junk.bin")
    with open(junk, "wb") as f:
        f.write(b"\0" * 256)
    with pytest.raises(MrhsError) as e:
        mrhs_load_setup(fresh.ctx, junk)
    assert e.value.status == MRHS_ERR_ARG

    # one flipped byte in the payload: checksum mismatch, and no setup afterwards
    bad = bytearray(data)
    bad[len(bad) // 2] ^= 0x5A
    damaged = str(tmp_path / "damaged.bin")
    with open(damaged, "wb") as f:
        f.write(bytes(bad))
    dst = make(prec)
    with pytest.raises(MrhsError) as e:
        mrhs_load_setup(dst.ctx, damaged)
    assert e.value.status == MRHS_ERR_ARG
    with pytest.raises(MrhsError) as e:
        dst.get_P()
    assert e.value.status == MRHS_ERR_STATE

    # truncated
    short = str(tmp_path / "short.bin")
    with open(short, "wb") as f:
        f.write(data[: len(data) - 1000])
    with pytest.raises(MrhsError) as e:
        mrhs_load_setup(dst.ctx, short)
    assert e.value.status == MRHS_ERR_ARG

    # the intact file still loads into the same context afterwards
    mrhs_load_setup(dst.ctx, path)
    assert np.array_equal(dst.get_Dc(), src.get_Dc())
    for lat in (fresh, src, other, dst):
        lat.close()
