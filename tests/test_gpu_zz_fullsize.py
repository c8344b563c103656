"""Parity at the full benchmark size: 48^3 x 96 lattice (10.6M sites), 4^4
domains, N_tv = 32 right-hand sides, FP32 setup, through the same calls and
launch configuration as the benchmark (bench.py's default workload).

The oracle cannot run the whole lattice in seconds, so the checks are:
  - the stencil on sampled sites (corners, the t boundary, random sites), each
    computed by the oracle from a 4^4 cut-out of the fields around it;
  - one SAP sweep from x0 = 0 on sampled colour-0 domains (including domains
    at the periodic and antiperiodic boundaries), each computed by the oracle
    from that domain's fields alone (tests/lattice_helpers.py; the cut-outs
    are proved against whole-lattice oracle runs in test_sampled_helpers.py);
  - P on every aggregate by properties that fix it at any size: the
    test vectors lie in range(P) (P P^dag v = v), R P = 1, and R v is upper
    triangular with a positive real diagonal, which makes P the unique Q
    factor of the thin QR of the test vectors;
  - D_c on every aggregate by its definition as a property: the coarse
    stencil equals R D P on random coarse vectors.
Sampled values are read from the device fields directly, at the device index
of each site (aggregate-major order; checked against pack/unpack first).
Needs about 220 GB of device memory and 10 GB of host memory.
"""
import os
import sys

import numpy as np
import pytest

import oracle
import paper_1601_03184_gb300 as pkg
from paper_1601_03184_gb300 import MRHS_F32, MRHS_PREC_FP32, Lattice, inputs
from lattice_helpers import cutout, device_site, lex, sap_sweep_on_domain, stencil_at_site

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402  (the benchmark's workload definition)

pytestmark = pytest.mark.gpu

CFG = bench.CONFIGS[bench.DEFAULT_CONFIG]
DIMS, AGG, N = tuple(CFG["dims"]), tuple(CFG["agg"]), int(CFG["ntv"])
V = int(np.prod(DIMS))
NAGG = int(np.prod([d // a for d, a in zip(DIMS, AGG)]))
M0, CSW = bench.load_m0(CFG["m0_keys"])[0], CFG["csw"]
N_MR = bench.SCHEDULE["init_mr"]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def gather(field, sites, dims=None, agg=None, nrhs=None):
    """[nrhs, len(sites), 12] complex128 values of a device FP32 field at
    canonical sites (default: the benchmark lattice)"""
    import torch

    dims, agg, nrhs = dims or DIMS, agg or AGG, nrhs or N
    vol = int(np.prod(dims))
    sd = device_site(dims, agg, np.asarray(sites))
    assert sd.min() >= 0 and sd.max() < vol
    f = field.view(torch.float32).view(vol, 12, 2, nrhs)
    g = f[torch.as_tensor(sd, dtype=torch.long, device=field.device)].double().cpu().numpy()
    return (g[:, :, 0, :] + 1j * g[:, :, 1, :]).transpose(2, 0, 1)


def test_device_order_read_back_small():
    """gather() reads what mrhs_pack wrote (small lattice, every site)"""
    dims, agg, nrhs = (8, 8, 8, 8), (4, 4, 4, 4), 4
    lat = Lattice(dims, agg, nrhs, MRHS_PREC_FP32)
    host = inputs.gaussian_field((nrhs, lat.V, 12), 71).astype(np.complex64)
    dev = lat.to_device(host, MRHS_F32)
    got = gather(dev, np.arange(lat.V), dims, agg, nrhs)
    assert np.array_equal(got, host.astype(np.complex128))
    lat.close()


@pytest.fixture(scope="module")
def full():
    import torch

    torch.cuda.empty_cache()
    free = torch.cuda.mem_get_info()[0]
    if free < 225e9:
        pytest.skip("the 48^3x96 check needs about 220 GB of free device memory (%.0f GB free)" % (free / 1e9))
    U = inputs.gauge_field(DIMS, CFG["eps"], CFG["gseed"], device="cuda")
    lat = Lattice(DIMS, AGG, N, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(M0, CSW)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(CFG["tvseed"])
    psi = torch.randn(pkg.mrhs_field_bytes(lat.ctx, N, MRHS_F32, 0) // 4, generator=gen, device="cuda",
                      dtype=torch.float32)
    yield dict(U=U, lat=lat, psi=psi)
    lat.close()
    del psi
    torch.cuda.empty_cache()


def test_tables_full_size(full):
    """the library's aggregate table gives the device order used by gather()"""
    _, aggof, _ = full["lat"].tables()
    s = np.random.default_rng(72).integers(0, V, 100000)
    assert np.array_equal(aggof[s, 0].astype(np.int64) * int(np.prod(AGG)) + aggof[s, 1], device_site(DIMS, AGG, s))


def test_stencil_full_size_sampled_sites(full):
    import torch

    lat, psi, U = full["lat"], full["psi"], full["U"]
    y = torch.empty_like(psi)
    lat.apply_D(psi, y, N, MRHS_F32)
    torch.cuda.synchronize()
    L = DIMS
    # corners, both sides of the t boundary, the middle, random sites
    sites = [0, V - 1, lex([0, 0, 0, L[3] - 1], L), lex([L[0] - 1, 0, L[2] - 1, 0], L),
             lex([L[0] // 3, L[1] - 1, L[2] // 9, 0], L), lex([3, L[1] - 1, 0, L[3] - 1], L),
             lex([L[0] // 2, L[1] // 2, L[2] // 2, L[3] // 2], L)]
    sites += [int(s) for s in np.random.default_rng(73).integers(0, V, 25)]
    got = gather(y, sites)
    for i, s in enumerate(sites):
        ref = stencil_at_site(DIMS, U, M0, CSW, lambda g: gather(psi, g), s)
        assert rel(got[:, i], ref) < 1e-5, s
    del y


def test_sap_sweep_full_size_sampled_domains(full):
    import torch

    lat, psi, U = full["lat"], full["psi"], full["U"]
    x = torch.zeros_like(psi)
    lat.sap(psi, x, N, MRHS_F32, 1, N_MR)
    torch.cuda.synchronize()
    nb = [d // a for d, a in zip(DIMS, AGG)]
    # the first and last domains, domains at the t boundary and inside; the
    # first coordinate is moved by one where needed to make the domain colour 0
    for b in [(0, 0, 0, 0), (0, 0, 0, nb[3] - 1), (nb[0] - 1, nb[1] - 1, nb[2] - 1, nb[3] - 1),
              (nb[0] // 2, nb[1] // 2, nb[2] // 2, nb[3] // 2), (0, nb[1] - 1, 0, nb[3] // 2)]:
        block = ((b[0] + sum(b) % 2) % nb[0],) + tuple(b[1:])
        assert sum(block) % 2 == 0  # colour 0: updated first
        ref, g = sap_sweep_on_domain(DIMS, AGG, U, M0, CSW, lambda s: gather(psi, s), block, N_MR)
        assert rel(gather(x, g), ref) < 1e-5, block
    del x
    pkg.mrhs_trim(lat.ctx)


def coarse_complex(field):
    """[nagg, 2N, N] complex128 view of a device FP32 coarse field
    (row h*N + i of aggregate A, right-hand side r)"""
    import torch

    f = field.view(NAGG, 2 * N, 2, N).double()
    return torch.complex(f[:, :, 0, :], f[:, :, 1, :])


def test_gram_schmidt_and_coarse_operator_full_size(full):
    import torch

    lat, psi = full["lat"], full["psi"]
    lat.set_tv(psi, MRHS_F32)
    lat.build_P()
    nc = pkg.mrhs_field_bytes(lat.ctx, N, MRHS_F32, 1) // 4
    vc = torch.empty(nc, device="cuda", dtype=torch.float32)
    lat.restrict(psi, vc, N, MRHS_F32)
    torch.cuda.synchronize()
    C = coarse_complex(vc)
    for h in range(2):
        T = C[:, h * N:(h + 1) * N, :]  # (P_{A,h}^dag v_r)_i
        col = T.abs().pow(2).sum(dim=1).sqrt()  # |v_r on A x h| when v_r lies in range(P)
        low = torch.tril(T, diagonal=-1).abs().amax(dim=1)
        assert float((low / col).max()) < 1e-4
        d = torch.diagonal(T, dim1=1, dim2=2)
        assert bool((d.real > 0).all())
        assert float((d.imag.abs() / d.real).max()) < 1e-4
    del C, T
    # v lies in range(P): P R v = v (fine fields are 32.6 GB: differences in
    # place, FP32 norms)
    u = torch.empty_like(psi)
    lat.prolong(vc, u, N, MRHS_F32)
    u.sub_(psi)
    assert float(torch.linalg.vector_norm(u) / torch.linalg.vector_norm(psi)) < 1e-5
    # R P = 1 on random coarse vectors
    gen = torch.Generator(device="cuda")
    gen.manual_seed(74)
    xc = torch.randn(nc, generator=gen, device="cuda", dtype=torch.float32)
    lat.prolong(xc, u, N, MRHS_F32)
    lat.restrict(u, vc, N, MRHS_F32)
    assert float(torch.linalg.vector_norm((vc - xc).double()) / torch.linalg.vector_norm(xc.double())) < 1e-5

    # D_c = R D P: the coarse stencil against restrict(D(prolong(xc)))
    lat.build_Dc()
    yc = torch.empty_like(xc)
    lat.apply_Dc(xc, yc, N, MRHS_F32)
    du = torch.empty_like(psi)
    lat.prolong(xc, u, N, MRHS_F32)
    lat.apply_D(u, du, N, MRHS_F32)
    lat.restrict(du, vc, N, MRHS_F32)
    torch.cuda.synchronize()
    assert float(torch.linalg.vector_norm((yc - vc).double()) / torch.linalg.vector_norm(vc.double())) < 1e-4
    del u, du
    pkg.mrhs_trim(lat.ctx)


def test_coarse_operator_full_size_against_oracle_cutouts(full):
    """The nine D_c blocks of sampled aggregates at full size against the
    oracle. A block of aggregate A involves only P on A and on its neighbour,
    the links between them and the clover term on A, and P on an aggregate is
    the thin-QR factor of the test vectors there: so the oracle's FP64
    Gram-Schmidt and coarse operator on the 12^4 cut-out of the fields around
    A (3^4 aggregates, A in the middle) give A's blocks exactly. The GPU's
    blocks are read column by column from the coarse stencil: x_c = e_j on
    the neighbour aggregate B and zero elsewhere gives column j of
    D_c[A][k] in y_c(A) (2 N_tv = 64 right-hand sides, one per column).
    Sampled aggregates: the middle of the lattice and one at x = 0 (periodic
    wrap in x); the t boundary is avoided (the cut-out has its own)."""
    import torch

    lat, psi, U = full["lat"], full["psi"], full["U"]
    lat.set_tv(psi, MRHS_F32)
    lat.build_P()
    lat.build_Dc()
    _, _, aggnbr = lat.tables()
    nb = [d // a for d, a in zip(DIMS, AGG)]
    nc = 2 * N
    ncb = pkg.mrhs_field_bytes(lat.ctx, nc, MRHS_F32, 1) // 4
    xc = torch.zeros(ncb, device="cuda", dtype=torch.float32)
    yc = torch.empty_like(xc)
    xv = xc.view(NAGG, nc, 2, nc)
    yv = yc.view(NAGG, nc, 2, nc)
    eye = torch.arange(nc, device="cuda")
    for b in [(nb[0] // 2, nb[1] // 2, nb[2] // 2, nb[3] // 2), (0, nb[1] - 1, 3, 5)]:
        A_ = int(lex(np.asarray(b), nb))
        gpu = np.zeros((9, nc, nc), np.complex128)
        for k in range(9):
            B = A_ if k == 0 else int(aggnbr[A_, k - 1])
            xc.zero_()
            xv[B, eye, 0, eye] = 1.0
            lat.apply_Dc(xc, yc, nc, MRHS_F32)
            blk = yv[A_].double().cpu().numpy()  # [i][re/im][column r]
            gpu[k] = blk[:, 0, :] + 1j * blk[:, 1, :]
        origin = np.asarray(b) * np.asarray(AGG)
        glob, wrapped = cutout(DIMS, origin - np.asarray(AGG), 3 * AGG[0])
        assert not wrapped.any()
        d12 = (3 * AGG[0],) * 4
        Uc = U[glob]
        Ac = oracle.clover(d12, Uc, M0, CSW)
        Pc = oracle.gram_schmidt(d12, AGG, gather(psi, glob))
        Dref = oracle.coarse_op(d12, AGG, Uc, Ac, Pc)[int(lex(np.array([1, 1, 1, 1]), (3, 3, 3, 3)))]
        for k in range(9):
            assert rel(gpu[k], Dref[k]) < 1e-5, (b, k, rel(gpu[k], Dref[k]))
    del xc, yc
    pkg.mrhs_trim(lat.ctx)
