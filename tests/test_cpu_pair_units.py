"""Host-only checks of the FP32 pair sum's work lists (swimmer_pair_units; no device work).

The pair sum evaluates each unordered pair of points once (Eq. BrV is even in the
separation d = X_i - X_j, so one kernel lookup serves both points).  A unit is 16 steps of a
warp: lane l holds target I*32 + l (and I2*32 + l in a two-target unit) and at step d meets
source J*32 + (l + d) mod 32.  Whatever the grouping, the lists must cover every unordered
pair of the nb*32 points exactly once and no point with itself; a two-target unit must name
three distinct blocks (its three partial sums go to three different rows).
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
    for I, J, d0, I2 in units:
        diag = I == J
        steps = range(1, 17) if diag else range(d0, d0 + 16)
        targets = [I] + ([] if I2 == 255 else [I2])
        for d in steps:
            for lane in range(32):
                if diag and d == 16 and lane >= 16:
                    continue  # lanes l and l + 16 meet the same pair at d = 16
                j = J * 32 + (lane + d) % 32
                for T in targets:
                    i = T * 32 + lane
                    seen[(min(i, j), max(i, j))] += 1
    return seen


@pytest.mark.parametrize("wide", [0, 1])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 6, 7, 8, 9, 13, 16, 31, 32])
def test_every_unordered_pair_once(api, nb, wide):
    units = api.swimmer_pair_units(nb, wide)
    e = nb * (nb - 1) // 2
    assert len(units) == (nb + 2 * ((e + 1) // 2) if wide else nb * nb)
    seen = _pairs(units)
    n = nb * 32
    assert all(i != j for i, j in seen), "a point met itself"
    assert len(seen) == n * (n - 1) // 2
    assert set(seen.values()) == {1}


@pytest.mark.parametrize("nb", list(range(1, 33)))
def test_wide_grouping(api, nb):
    units = api.swimmer_pair_units(nb, 1)
    wide = [u for u in units if u[3] != 255]
    single = [u for u in units if u[3] == 255 and u[0] != u[1]]
    e = nb * (nb - 1) // 2
    assert len(wide) == 2 * (e // 2) and len(single) == 2 * (e % 2)
    for I, J, d0, I2 in wide:
        assert len({I, J, I2}) == 3 and d0 in (0, 16)
    # each unit's two halves (d0 = 0 and 16) come together
    for k in range(0, len(wide), 2):
        assert wide[k][:2] + wide[k][3:] == wide[k + 1][:2] + wide[k + 1][3:]
        assert (wide[k][2], wide[k + 1][2]) == (0, 16)
    assert all(0 <= b < nb for u in units for b in (u[0], u[1]))


def test_rejects_bad_arguments(api):
    for nb, wide in ((0, 0), (33, 0), (4, 2)):
        with pytest.raises(Exception):
            api.swimmer_pair_units(nb, wide)
