"""Host-only checks of the pre-fetch decision tree that tmcmc_stage evaluates for each live
chain (tmcmc_tree_template; no device work).  The tree must be a valid binary decision
tree rooted at the chain's next step, and it must hold the most probable nodes: for an
acceptance probability p, a node's probability is the product of p (accept edges) and
1 - p (reject edges) along its path, and a best-first tree of M nodes contains the M most
probable nodes of the infinite decision tree whose ancestors it contains."""
import os

import pytest

from paper_1910_12007_gb300 import _lib


@pytest.fixture(scope="module")
def api():
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    from paper_1910_12007_gb300 import api as a

    return a


def _prob(nodes, v, p):
    pr = 1.0
    while nodes[v][0] >= 0:
        pr *= p if nodes[v][2] else 1.0 - p
        v = nodes[v][0]
    return pr


@pytest.mark.parametrize("M,p,cap", [(1, 0.8, 31), (2, 0.8, 31), (7, 0.5, 31), (63, 0.5, 31), (200, 0.86, 31),
                                     (1024, 0.86, 12), (1024, 0.3, 31), (50, 0.9, 3), (300, 0.6, 8)])
def test_tree_is_a_valid_best_first_decision_tree(api, M, p, cap):
    nodes = api.tmcmc_tree_template(M, p, cap)
    n = len(nodes)
    assert 1 <= n <= M
    assert nodes[0][0] == -1 and nodes[0][1] == 0
    for v, (par, depth, is_acc, ac, rc) in enumerate(nodes):
        assert depth < cap
        if v:
            assert 0 <= par < v  # parents come first
            assert depth == nodes[par][1] + 1
            assert (nodes[par][3] if is_acc else nodes[par][4]) == v
        for ch, want in ((ac, 1), (rc, 0)):
            if ch >= 0:
                assert ch > v and nodes[ch][0] == v and nodes[ch][2] == want
    probs = [_prob(nodes, v, p) for v in range(n)]
    # best-first: probabilities never increase along the construction order
    assert all(probs[i + 1] <= probs[i] * (1 + 1e-12) for i in range(1, n - 1))
    # no missing child inside the depth cap is more probable than a chosen node
    frontier = [probs[v] * (p if ch == nodes[v][3] else 1 - p)
                for v in range(n) for ch in (nodes[v][3], nodes[v][4])
                if ch < 0 and nodes[v][1] + 1 < cap]
    if n > 1 and frontier:
        assert max(frontier) <= min(probs[1:]) * (1 + 1e-12)
    if n < M:  # stopped early only because the depth cap ran out: complete tree
        assert n == 2 ** cap - 1


def test_tree_shapes_with_known_answers(api):
    # p = 1/2: every level is equally likely, so 2^(k+1) - 1 nodes form the complete tree
    nodes = api.tmcmc_tree_template(7, 0.5, 31)
    assert sorted(d for _, d, _, _, _ in nodes) == [0, 1, 1, 2, 2, 2, 2]
    # a likely acceptance: the first nodes follow the all-accept path (0.86^k > 0.14)
    nodes = api.tmcmc_tree_template(5, 0.86, 31)
    assert [d for _, d, _, _, _ in nodes] == [0, 1, 2, 3, 4]
    assert all(a == 1 for _, _, a, _, _ in nodes[1:])
    # rare acceptance: the all-reject path
    nodes = api.tmcmc_tree_template(4, 0.1, 31)
    assert [(d, a) for _, d, a, _, _ in nodes] == [(0, 0), (1, 0), (2, 0), (3, 0)]
    # the cap truncates the tree
    assert len(api.tmcmc_tree_template(100, 0.5, 2)) == 3


def test_tree_rejects_bad_arguments(api):
    for args in [(0, 0.5, 4), (4, 0.0, 4), (4, 1.0, 4), (4, 0.5, 0), (4, 0.5, 32)]:
        with pytest.raises(RuntimeError):
            api.tmcmc_tree_template(*args)
