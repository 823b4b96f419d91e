"""Host-side helpers of the learned path: the offset calibration and the per-popcount quantile table
(the non-learned predictor the MLP is compared with).  Values are checked against direct definitions
on small hand-built inputs."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def learn():
    import __graft_entry__ as ge

    ge._cuda_build_module().build()
    from paper_1906_06170_gb300 import learn as mod

    return mod


def packed_with_popcounts(pcs):
    """One packed query per requested popcount: the lowest bits set (bit j = word j/64, bit j%64)."""
    out = np.zeros((len(pcs), 3), np.uint64)
    for r, p in enumerate(pcs):
        for j in range(p):
            out[r, j // 64] |= np.uint64(1) << np.uint64(j % 64)
    return out


def test_query_popcounts(learn):
    pcs = [0, 1, 63, 64, 65, 127, 128, 166]
    assert learn.query_popcounts(packed_with_popcounts(pcs)).tolist() == pcs


def test_popc_table_quantiles_and_nearest_fill(learn):
    pcs = [10] * 5 + [20] * 3
    t = np.array([1, 2, 3, 4, 5, 7, 9, 11], np.float64)
    table = learn.popc_quantile_table(packed_with_popcounts(pcs), t, 0.5)
    assert table.shape == (167,)
    assert table[10] == pytest.approx(np.quantile([1, 2, 3, 4, 5], 0.5))
    assert table[20] == pytest.approx(np.quantile([7, 9, 11], 0.5))
    assert table[0] == table[10] and table[14] == table[10] and table[16] == table[20] and table[166] == table[20]
    tau = learn.table_tau(table, packed_with_popcounts([10, 20, 3]), offset=1.0)
    assert tau.dtype == np.float32 and tau.tolist() == [table[10] + 1, table[20] + 1, table[10] + 1]


def test_offset_for_is_the_smallest_sufficient_shift(learn):
    pred = np.array([10.0, 20.0, 30.0, 40.0])
    t = np.array([12.0, 20.0, 29.0, 45.0])
    # ceil(pred + d) < t must hold for no query: the worst shortfall is 45 - 40 = 5
    assert learn.offset_for(pred, t, 0.0) == 5.0
    # one query of four may fall short: the second worst is 12 - 10 = 2
    assert learn.offset_for(pred, t, 0.25) == 2.0
