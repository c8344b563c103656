"""The cut-out helpers behind the sampled full-size GPU checks, proved on the
CPU against the oracle on whole small lattices: the operator at single sites
(including sites whose hops cross the antiperiodic t boundary) and one SAP
sweep from x0 = 0 on single colour-0 domains (including domains next to the
t boundary)."""
import numpy as np

import oracle
from paper_1601_03184_gb300 import inputs
from lattice_helpers import device_site, lex, sap_sweep_on_domain, stencil_at_site, vol


def test_stencil_at_site_equals_the_whole_lattice_operator():
    dims, m0, csw = (6, 4, 8, 6), -0.3, 1.7
    U = inputs.gauge_field(dims, 0.6, 31)
    A = oracle.clover(dims, U, m0, csw)
    psi = inputs.gaussian_field((3, vol(dims), 12), 32)
    ref = oracle.apply_D(dims, U, A, psi)
    rng = np.random.default_rng(33)
    sites = [0, vol(dims) - 1, lex([0, 0, 0, 5], dims), lex([5, 3, 7, 0], dims), lex([2, 1, 4, 3], dims)]
    sites += list(rng.integers(0, vol(dims), 10))
    for s in sites:
        got = stencil_at_site(dims, U, m0, csw, lambda g: psi[:, g], s)
        assert np.abs(got - ref[:, s]).max() < 1e-13 * np.abs(ref[:, s]).max(), s


def test_sap_sweep_on_domain_equals_the_whole_lattice_sweep():
    dims, agg, m0, csw, n_mr = (8, 8, 8, 16), (4, 4, 4, 4), -0.3, 1.7, 4
    U = inputs.gauge_field(dims, 0.6, 34)
    A = oracle.clover(dims, U, m0, csw)
    b = inputs.gaussian_field((2, vol(dims), 12), 35)
    ref = oracle.sap(dims, agg, U, A, b, np.zeros_like(b), 1, n_mr)
    for block in [(0, 0, 0, 0), (1, 0, 0, 3), (0, 1, 1, 2), (1, 1, 1, 1)]:
        assert sum(block) % 2 == 0
        got, g = sap_sweep_on_domain(dims, agg, U, m0, csw, lambda s: b[:, s], block, n_mr)
        assert np.abs(got - ref[:, g]).max() < 1e-12 * np.abs(ref[:, g]).max(), block


def test_device_site_is_the_aggregate_major_order():
    dims, agg = (4, 6, 4, 8), (2, 3, 2, 2)
    _, aggof, _ = oracle.tables(dims, agg)
    s = np.arange(vol(dims))
    assert np.array_equal(device_site(dims, agg, s), aggof[:, 0] * int(np.prod(agg)) + aggof[:, 1])
    assert np.array_equal(np.sort(device_site(dims, agg, s)), s)
