"""The autotuner's host logic, without a GPU: the solver rule on measurements and the process-wide
cache keyed by device, Krylov precision, preconditioner and model size class."""
import pytest

from paper_2008_01539_gb300 import build as _build
from paper_2008_01539_gb300 import lns


@pytest.fixture(scope="module", autouse=True)
def lib():
    _build.build()
    lns._lib = None
    return lns.load()


def test_pick_takes_the_largest_size_of_the_winning_prefix():
    sizes = [500, 1000, 2000, 4000, 8000]
    # cluster faster up to 2000, slower at 4000, faster again at 8000: the prefix stops at 2000
    assert lns.lns_tune_pick(sizes, [1, 2, 3, 9, 5], [2, 3, 4, 8, 9]) == 2000
    assert lns.lns_tune_pick(sizes, [1, 1, 1, 1, 1], [2, 2, 2, 2, 2]) == 8000
    assert lns.lns_tune_pick(sizes, [3, 1, 1, 1, 1], [2, 2, 2, 2, 2]) == 0
    # a system that did not fit the cluster solver (negative time) ends the prefix
    assert lns.lns_tune_pick(sizes, [1, 1, -1, 1, 1], [2, 2, 2, 2, 2]) == 1000
    # ties go to the grid solver
    assert lns.lns_tune_pick(sizes, [2, 2, 2, 2, 2], [2, 2, 2, 2, 2]) == 0
    assert lns.lns_tune_pick([], [], []) == 0


def test_cache_is_keyed_by_device_precision_preconditioner_and_size_class():
    lns.lns_tune_cache_clear()
    assert lns.lns_tune_cache(0, 1, 0, 166_659) is None
    lns.lns_tune_cache_store(0, 1, 0, 166_659, cluster_max_rows=2048, asm_block=128, asm_blocks_per_sm=8,
                             set_blocks_per_sm=2, measured=1)
    got = lns.lns_tune_cache(0, 1, 0, 166_659)
    assert got == dict(cluster_max_rows=2048, asm_block=128, asm_blocks_per_sm=8, set_blocks_per_sm=2, measured=1)
    # same bit length of n_cells (2^17 <= n < 2^18): same class
    assert lns.lns_tune_cache(0, 1, 0, 131_072) == got and lns.lns_tune_cache(0, 1, 0, 262_143) == got
    # other class, device, precision or preconditioner: no entry
    assert lns.lns_tune_cache(0, 1, 0, 262_144) is None
    assert lns.lns_tune_cache(0, 1, 0, 131_071) is None
    assert lns.lns_tune_cache(1, 1, 0, 166_659) is None
    assert lns.lns_tune_cache(0, 0, 0, 166_659) is None
    assert lns.lns_tune_cache(0, 1, 1, 166_659) is None
    lns.lns_tune_cache_store(0, 1, 0, 170_000, cluster_max_rows=0, asm_block=64, asm_blocks_per_sm=4,
                             set_blocks_per_sm=4, measured=1)
    assert lns.lns_tune_cache(0, 1, 0, 166_659)["cluster_max_rows"] == 0  # replaced
    lns.lns_tune_cache_clear()
    assert lns.lns_tune_cache(0, 1, 0, 166_659) is None
