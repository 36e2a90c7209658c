"""Pins for the oracle's reverse Cuthill-McKee order (Sec. III)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order, connected_components, reverse_cuthill_mckee

from oracle.liouvillian import Params, augmented, bandwidth_profile, liouvillian, symmetric_pattern
from oracle.reorder_factor import permute_symmetric, rcm_permutation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def random_graph(rng, n, p):
    M = sp.random(n, n, density=p, random_state=rng, format="csr")
    M = M + sp.identity(n)
    return sp.csr_matrix(M, dtype=np.complex128)


def check_cm_properties(A, perm):
    """Check, on the CM order (perm reversed), what the paper's description
    fixes: a BFS per connected component that starts at a node of minimum
    (degree, index), whose nodes appear level by level; each node is placed
    by its earliest-placed neighbour; siblings are in (degree, index) order."""
    S = symmetric_pattern(A)
    n = S.shape[0]
    deg = np.diff(S.indptr)
    cm = np.asarray(perm)[::-1]
    assert sorted(cm.tolist()) == list(range(n))
    pos = np.empty(n, dtype=np.int64)
    pos[cm] = np.arange(n)
    ncomp, label = connected_components(S, directed=False)
    starts = []
    for idx, v in enumerate(cm):
        nbrs = S.indices[S.indptr[v]:S.indptr[v + 1]]
        earlier = [u for u in nbrs if pos[u] < idx]
        if not earlier:
            starts.append(v)
            # start node: min (degree, index) among the nodes still unplaced
            remaining = cm[idx:]
            key = min((deg[u], u) for u in remaining)
            assert (deg[v], v) == key
    assert len(starts) == ncomp
    # BFS levels from each start are non-decreasing along the order
    for s in starts:
        comp = np.where(label == label[s])[0]
        order, pred = breadth_first_order(S, s, directed=False, return_predecessors=True)
        dist = np.zeros(n, dtype=np.int64)
        for v in order[1:]:
            dist[v] = dist[pred[v]] + 1
        seq = sorted(comp, key=lambda v: pos[v])
        d = [dist[v] for v in seq]
        assert d == sorted(d)
    # parent = earliest-placed neighbour; children of one parent sorted by (degree, index)
    parent = {}
    for v in cm:
        nbrs = S.indices[S.indptr[v]:S.indptr[v + 1]]
        earlier = [u for u in nbrs if pos[u] < pos[v]]
        if earlier:
            parent[v] = min(earlier, key=lambda u: pos[u])
    kids = {}
    for v in cm:
        if v in parent:
            kids.setdefault(parent[v], []).append(v)
    for u, ch in kids.items():
        assert ch == sorted(ch, key=lambda v: (deg[v], v))
        # siblings are contiguous and follow the parent's earlier siblings' children
        ps = [pos[v] for v in ch]
        assert ps == list(range(ps[0], ps[0] + len(ps)))
    return True


@pytest.mark.parametrize("seed", range(8))
def test_cm_properties_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 40))
    A = random_graph(rng, n, float(rng.uniform(0.03, 0.2)))
    perm = rcm_permutation(A)
    check_cm_properties(A, perm)


def test_cm_properties_liouvillian():
    p = Params(3, 5, **TINY)
    Lt, *_ = augmented(p, "replace")
    check_cm_properties(Lt, rcm_permutation(Lt))


def test_path_graph_is_reversed_path():
    """A path 0-1-...-k: lowest degree start is node 0 (degree 2 with the
    diagonal, index 0), CM is 0..k and RCM is k..0."""
    k = 9
    A = sp.diags([np.ones(k), np.ones(k + 1), np.ones(k)], [-1, 0, 1], format="csr", dtype=complex)
    np.testing.assert_array_equal(rcm_permutation(A), np.arange(k, -1, -1))


def test_components_and_isolated_nodes():
    A = sp.csr_matrix(np.array([[1, 1, 0, 0, 0],
                                [1, 1, 0, 0, 0],
                                [0, 0, 1, 0, 0],
                                [0, 0, 0, 1, 1],
                                [0, 0, 0, 1, 1]], dtype=complex))
    perm = rcm_permutation(A)
    # degrees 2,2,1,2,2: start at node 2 (component {2}), then {0,1}, then {3,4}
    np.testing.assert_array_equal(perm[::-1], [2, 0, 1, 3, 4])


@pytest.mark.parametrize("Nc,Nm", [(3, 5), (6, 20)])
def test_equals_library_rcm_where_ties_agree(Nc, Nm):
    """At these sizes SciPy's RCM breaks ties the same way; the orders agree."""
    p = Params(Nc, Nm, **TINY)
    Lt, *_ = augmented(p, "replace")
    S = symmetric_pattern(Lt)
    ref = reverse_cuthill_mckee(S, symmetric_mode=True)
    np.testing.assert_array_equal(rcm_permutation(Lt), ref)


def test_reduction_factors_fig1():
    """Fig. 1: RCM lowers B about 5x and P about 2.5x at N_c = 4, N_m = 8;
    Sec. III: B and P of L~_RCM fall below those of L itself."""
    g = json.load(open(os.path.join(GOLDEN, "paper_fig1.json")))
    p = Params(g["Nc"], g["Nm"], **TINY)
    Lt, *_ = augmented(p, g["trace_mode"])
    A = permute_symmetric(Lt, rcm_permutation(Lt))
    b0, b1 = bandwidth_profile(Lt), bandwidth_profile(A)
    rB, rP = b0["B"] / b1["B"], b0["P"] / b1["P"]
    assert 4.0 < rB < 6.5, rB
    assert 2.0 < rP < 3.0, rP
    bl = bandwidth_profile(liouvillian(p))
    assert b1["B"] < bl["B"] and b1["P"] < bl["P"]


def test_permute_symmetric_definition():
    rng = np.random.default_rng(3)
    A = random_graph(rng, 12, 0.2).toarray() * (1 + 1j)
    perm = rng.permutation(12).astype(np.int32)
    B = permute_symmetric(sp.csr_matrix(A), perm).toarray()
    for r in range(12):
        for c in range(12):
            assert B[r, c] == A[perm[r], perm[c]]
