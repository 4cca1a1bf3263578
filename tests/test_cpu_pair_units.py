"""Host-only checks of the FP32 pair sum's work lists (swimmer_pair_units; no device work).

The pair sum evaluates each unordered pair of points once (Eq. BrV is even in the
separation d = X_i - X_j, so one kernel lookup serves both points).  A unit is 16 steps of a
warp: lane l holds target I*32 + l for each of its 1, 2 or 4 target blocks I and at step d
meets source J*32 + (l + d) mod 32.  Whatever the grouping, the lists must cover every
unordered pair of the nb*32 points exactly once and no point with itself; a multi-target
unit must name distinct blocks (its partial sums go to different rows).
"""
import os
from collections import Counter

import pytest

from paper_1910_12007_gb300 import _lib


@pytest.fixture(scope="module")
def api():
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    from paper_1910_12007_gb300 import api as a

    return a


def _pairs(units):
    """Unordered point pairs each unit evaluates, by simulating the warp's walk."""
    seen = Counter()
    for targets, J, d0 in units:
        diag = d0 == 1
        steps = range(1, 17) if diag else range(d0, d0 + 16)
        for d in steps:
            for lane in range(32):
                if diag and d == 16 and lane >= 16:
                    continue  # lanes l and l + 16 meet the same pair at d = 16
                j = J * 32 + (lane + d) % 32
                for T in targets:
                    i = T * 32 + lane
                    seen[(min(i, j), max(i, j))] += 1
    return seen


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 6, 7, 8, 9, 13, 16, 31, 32])
def test_every_unordered_pair_once(api, nb, mode):
    units = api.swimmer_pair_units(nb, mode)
    assert len(units) <= nb * nb
    if mode == 0:
        assert len(units) == nb * nb
    seen = _pairs(units)
    n = nb * 32
    assert all(i != j for i, j in seen), "a point met itself"
    assert len(seen) == n * (n - 1) // 2
    assert set(seen.values()) == {1}


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("nb", list(range(1, 33)))
def test_grouping(api, nb, mode):
    units = api.swimmer_pair_units(nb, mode)
    off = [u for u in units if u[2] != 1]
    e = nb * (nb - 1) // 2
    singles = [u for u in off if len(u[0]) == 1]
    if mode == 1:
        assert len(singles) == 2 * (e % 2)  # at most one block pair stays alone
        assert all(len(u[0]) in (1, 2) for u in off)
    elif nb < 8:
        # too few blocks for four-target units: the two-target list
        assert units == api.swimmer_pair_units(nb, 1)
    else:
        # four-target units carry nearly every block pair
        assert len(singles) <= 4
        quads = [u for u in off if len(u[0]) == 4]
        assert 4 * len(quads) // 2 >= 0.9 * e
    for targets, J, d0 in off:
        assert len(set(targets) | {J}) == len(targets) + 1 and d0 in (0, 16)
    # each unit's two halves (d0 = 0 and 16) come together
    for k in range(0, len(off), 2):
        assert off[k][:2] == off[k + 1][:2] and (off[k][2], off[k + 1][2]) == (0, 16)
    assert all(0 <= b < nb for u in units for b in u[0] + (u[1],))
    assert [u for u in units if u[2] == 1] == [((i,), i, 1) for i in range(nb)]


def test_rejects_bad_arguments(api):
    for nb, mode in ((0, 0), (33, 0), (4, 3), (4, -1)):
        with pytest.raises(Exception):
            api.swimmer_pair_units(nb, mode)
