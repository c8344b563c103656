"""The training and judging protocol of the learned generator
(paper_1601_03184_gb300/learned_protocol.py) on a reduced case: 8^4 lattice,
4^4 domains, 8 test vectors, the 4 -> 32 -> 32 -> 4 network, three training
fields of roughness in [0.4, 0.7] and one unseen field. The full protocol
(64 fields at 16^3 x 32, N_tv = 20, 8 unseen fields) is a separate run; this
test checks that the protocol runs end to end through the C ABI, that
training lowers the loss, that both setups converge, and that the learned
initial phase (one SAP sweep + network) gives test vectors with a lower
Rayleigh quotient than the network's input has (the gain of the network)."""
import numpy as np
import pytest

from paper_1601_03184_gb300 import learned_protocol

pytestmark = pytest.mark.gpu


def test_protocol_reduced():
    res = learned_protocol.run(n_train=3, n_test=1, dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8,
                               widths=(4, 32, 32, 4), steps=20, lr=3e-3, m0_table={0.55: -0.3},
                               schedule=dict(n_refine=1, cmaxit=200), log=print)
    assert res["loss_last"] < res["loss_first"]
    t = res["tests"][0]
    for form in ("plain", "learned"):
        assert t[form]["relres"] <= 1e-10
        assert np.isfinite(t[form]["rq_init"]) and t[form]["rq_final"] <= t[form]["rq_init"] * 1.5
    assert t["learned"]["rq_init"] < t["learned"]["rq_one_sweep"]
