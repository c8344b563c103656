"""Host logic of the learned-generator protocol (no GPU): the seeded field
roughness draws, the m0 interpolation between the tuned proxy points, and the
table read from tests/golden/m0.json."""
import numpy as np

from paper_1601_03184_gb300 import learned_protocol as lp


def test_roughness_draws_are_seeded_and_in_range():
    a = lp.roughness(lp.TRAIN_SEED0, 64)
    b = lp.roughness(lp.TRAIN_SEED0, 64)
    t = lp.roughness(lp.TEST_SEED0, 8)
    assert np.array_equal(a, b)
    assert a.min() >= 0.4 and a.max() <= 0.7 and t.min() >= 0.4 and t.max() <= 0.7
    assert not np.array_equal(a[:8], t)  # unseen fields differ from the training ones


def test_m0_interpolation():
    table = {0.4: -0.3, 0.6: -0.6, 0.7: -0.9}
    assert lp.m0_for(0.4, table) == -0.3
    assert lp.m0_for(0.7, table) == -0.9
    assert abs(lp.m0_for(0.5, table) + 0.45) < 1e-12
    assert abs(lp.m0_for(0.65, table) + 0.75) < 1e-12
    # constant outside the tuned range
    assert lp.m0_for(0.3, table) == -0.3 and lp.m0_for(0.8, table) == -0.9


def test_m0_table_from_the_tuned_proxies():
    table = lp.load_m0_table(1.5)
    assert sorted(table) == [0.4, 0.6, 0.7]
    # rougher fields need a more negative bare mass to stay near critical
    assert table[0.4] > table[0.6] > table[0.7]
    assert lp.load_m0_table(1.7) and 0.6 in lp.load_m0_table(1.7)
