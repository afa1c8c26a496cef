"""Cases of the split rule (Sec. 3: the sub-elements replacing a split element)
for the host and device tests of the CUDA path's rule against the oracle.

A case is an element's four node indices, their creation ids, a side mask and
the new nodes on its cut edges (storage index and creation id, for every
(x, y) pair of local nodes, attached to x).  Storage indices are drawn apart
from creation ids, as they are after a node renumbering, so a rule that mixed
the two up would fail.  The expected sub-elements come from
oracle.sub_tet_nodes on creation ids and are mapped to storage indices.
"""
import numpy as np

from oracle.cem_oracle import sub_tet_nodes


def _case(conn_ids, mask, M, to_sto):
    """Arrays of one case: conn_ids (4 creation ids), M(id_x, id_y) the new node's id."""
    mn = -np.ones((4, 4), np.int64)
    mi = -np.ones((4, 4), np.int64)
    for x in range(4):
        for y in range(4):
            if x != y and ((mask >> x) & 1) != ((mask >> y) & 1):
                mi[x, y] = M(conn_ids[x], conn_ids[y])
                mn[x, y] = to_sto(mi[x, y])
    want = [[to_sto(v) for v in t] for t in sub_tet_nodes(conn_ids, mask, M)]
    return [to_sto(v) for v in conn_ids], list(conn_ids), mask, mn, mi, want


def _stack(cases):
    nodes = np.array([c[0] for c in cases], np.int64)
    ids = np.array([c[1] for c in cases], np.int64)
    mask = np.array([c[2] for c in cases], np.int64)
    mn = np.array([c[3] for c in cases], np.int64)
    mi = np.array([c[4] for c in cases], np.int64)
    return nodes, ids, mask, mn, mi, [c[5] for c in cases]


def random_cases(n, seed):
    """n elements with random ids, every side mask 1..14, storage ids a random permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(1 << 20)
    cases = []
    for q in range(n):
        ids = [int(v) for v in rng.choice(1 << 19, size=4, replace=False)]
        mask = 1 + q % 14
        new = {}
        nxt = iter(int(v) for v in (1 << 19) + rng.choice(1 << 19, size=16, replace=False))

        def M(a, b):
            if (a, b) not in new:
                new[(a, b)] = next(nxt)
            return new[(a, b)]
        cases.append(_case(ids, mask, M, lambda v: int(perm[v])))
    return _stack(cases)


def notch_cases(oracle, seed):
    """The notch splits of an oracle context (its node ids are creation ids)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(oracle.X.shape[0])
    cases = []
    for t, _step, _pattern, mask, _G in oracle.crack_state():
        conn_ids = [int(v) for v in oracle.conn[t]]
        cases.append(_case(conn_ids, int(mask), oracle._M, lambda v: int(perm[v])))
    return _stack(cases)
