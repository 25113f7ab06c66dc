"""Host logic of the MBIR module: the ordered-subset partition."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
pytest.importorskip("torch")
from paper_2503_16741_gb300.mbir import ordered_subsets  # noqa: E402


@pytest.mark.parametrize("nview,S", [(1, 1), (10, 3), (360, 10), (23, 23), (7, 2)])
def test_ordered_subsets_partition_the_views(nview, S):
    subs = ordered_subsets(nview, S)
    assert len(subs) == S
    flat = sorted(v for s in subs for v in s)
    assert flat == list(range(nview))  # every view exactly once
    for s, views in enumerate(subs):  # interleaved: s, s + S, s + 2S, ...
        assert views == list(range(s, nview, S))
    sizes = [len(s) for s in subs]
    assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("nview,S", [(5, 0), (5, 6)])
def test_ordered_subsets_reject_bad_counts(nview, S):
    with pytest.raises(ValueError):
        ordered_subsets(nview, S)
