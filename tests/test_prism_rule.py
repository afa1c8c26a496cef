"""The prism division of the split rule (Sec. 3) on both sides, no GPU.

The CUDA path's division (csrc/cem_prism.cuh, compiled here for the host) must
give the oracle's three tetrahedra for any prism: diagonals fixed by creation
ids, sub-elements named by storage ids.  Each quadrilateral face is cut along
the diagonal through its smallest id, which is what makes two split neighbours
cut their shared face alike; the oracle's division is pinned to that property,
to tiling the prism, and to conformity on a split mesh.
"""
import collections
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.cem_oracle import prism_tets

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2508_04076_gb300", "csrc", "cem_prism.cuh")

DRIVER = r"""
#include <cstdio>
#include "%s"
int main() {
    int A[3], B[3], Ae[3], Be[3], out[3][4];
    while (std::scanf("%%d %%d %%d %%d %%d %%d %%d %%d %%d %%d %%d %%d", &A[0], &A[1], &A[2], &B[0], &B[1], &B[2],
                      &Ae[0], &Ae[1], &Ae[2], &Be[0], &Be[1], &Be[2]) == 12) {
        cem_prism_division(A, B, Ae, Be, out);
        for (int r = 0; r < 3; ++r) std::printf("%%d %%d %%d %%d ", out[r][0], out[r][1], out[r][2], out[r][3]);
        std::printf("\n");
    }
    return 0;
}
"""


def _quad_diagonals(tets, A, B):
    """The diagonal each quadrilateral face of prism A/B gets from the tetrahedra."""
    edges = {frozenset(e) for t in tets for e in itertools.combinations(t, 2)}
    out = []
    for i in range(3):
        j = (i + 1) % 3
        d1, d2 = frozenset((A[i], B[j])), frozenset((A[j], B[i]))
        assert (d1 in edges) != (d2 in edges), "a quadrilateral face must be cut by exactly one diagonal"
        out.append(d1 if d1 in edges else d2)
    return out


def test_oracle_division_cuts_each_face_through_its_smallest_id():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        ids = rng.choice(1000, size=6, replace=False)
        A, B = tuple(int(x) for x in ids[:3]), tuple(int(x) for x in ids[3:])
        tets = prism_tets(A, B)
        assert len(tets) == 3 and all(len(set(t)) == 4 for t in tets)
        for i, diag in enumerate(_quad_diagonals(tets, A, B)):
            j = (i + 1) % 3
            assert min(A[i], A[j], B[i], B[j]) in diag


def test_oracle_division_tiles_the_prism():
    rng = np.random.default_rng(6)
    for _ in range(500):
        base = rng.standard_normal((3, 3))
        top = base + np.array([0.0, 0.0, 2.0]) + 0.5 * rng.standard_normal(3)   # planar (parallelogram) sides
        ids = rng.choice(100, size=6, replace=False)
        pos = {int(ids[k]): (base[k] if k < 3 else top[k - 3]) for k in range(6)}
        A, B = tuple(int(x) for x in ids[:3]), tuple(int(x) for x in ids[3:])
        vols = [abs(np.linalg.det(np.array([pos[t[1]] - pos[t[0]], pos[t[2]] - pos[t[0]], pos[t[3]] - pos[t[0]]])))
                / 6.0 for t in prism_tets(A, B)]
        # the prism's volume: its planar boundary triangulated, as cones from the top centroid
        c = top.mean(axis=0)
        ref = 0.0
        tris = [(base[0], base[1], base[2])]
        for i in range(3):
            j = (i + 1) % 3
            tris += [(base[i], base[j], top[j]), (base[i], top[j], top[i])]
        for a, b, d in tris:
            ref += abs(np.linalg.det(np.array([a - c, b - c, d - c]))) / 6.0
        assert min(vols) > 0.0
        assert abs(sum(vols) - ref) <= 1e-9 * ref


def test_split_neighbours_share_their_triangulation():
    from cem_inputs import kuhn_block
    from oracle import CEMOracle
    w = kuhn_block(16, 8, 2, 0.08, 0.04, 0.01, notch_length=0.04, traction=2.5e6)
    o = CEMOracle.from_workload(w)
    o.step(400)
    T0 = w.n_tets
    owners = collections.defaultdict(list)
    for t in range(T0):
        for f in range(4):
            owners[tuple(sorted(int(o.conn[t][l]) for l in range(4) if l != f))].append(t)
    subs = collections.defaultdict(list)
    for j in range(T0, o.conn.shape[0]):
        if o.active[j]:
            subs[int(o.parent[j])].append(j)

    def on_face(F, p):
        P = o.X[list(F)]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        n /= np.linalg.norm(n)
        tris = set()
        for j in subs[p]:
            for f in range(4):
                tri = [int(o.conn[j][l]) for l in range(4) if l != f]
                if np.all(np.abs((o.X[tri] - P[0]) @ n) < 1e-12):
                    tris.add(tuple(sorted(tri)))
        return tris

    shared = [(F, ts) for F, ts in owners.items() if len(ts) == 2 and o.side[ts[0]] and o.side[ts[1]]]
    assert len(shared) > 50
    for F, (p, q) in shared:
        assert on_face(F, p) == on_face(F, q), F


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_cuda_division_matches_the_oracle(tmp_path):
    src = tmp_path / "prism.cpp"
    src.write_text(DRIVER % HEADER)
    exe = tmp_path / "prism"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True, capture_output=True)
    rng = np.random.default_rng(7)
    cases, lines = [], []
    for _ in range(3000):
        ext = rng.choice(10**6, size=6, replace=False)          # creation ids
        sto = rng.choice(10**6, size=6, replace=False)          # storage indices
        cases.append((sto, ext))
        lines.append(" ".join(str(int(x)) for x in list(sto) + list(ext)))
    r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    rows = r.stdout.strip().split("\n")
    assert len(rows) == len(cases)
    for (sto, ext), row in zip(cases, rows):
        got = np.array(row.split(), dtype=np.int64).reshape(3, 4)
        to_sto = dict(zip((int(x) for x in ext), (int(x) for x in sto)))
        want = [[to_sto[v] for v in t] for t in prism_tets(tuple(int(x) for x in ext[:3]),
                                                           tuple(int(x) for x in ext[3:]))]
        assert got.tolist() == want


RULE_DRIVER = r"""
#include <cstdio>
#include "%s"
struct Table {
    const int* mn;
    const int* mi;
    void operator()(int x, int y, int* node, int* id) const {
        *node = mn[4 * x + y];
        *id = mi[4 * x + y];
    }
};
int main() {
    int nd[4], id[4], m, mn[16], mi[16], out[6][4];
    while (std::scanf("%%d %%d %%d %%d %%d %%d %%d %%d %%d", &nd[0], &nd[1], &nd[2], &nd[3], &id[0], &id[1], &id[2],
                      &id[3], &m) == 9) {
        for (int q = 0; q < 16; ++q) std::scanf("%%d", &mn[q]);
        for (int q = 0; q < 16; ++q) std::scanf("%%d", &mi[q]);
        const int k = cem_split_subs(nd[0], nd[1], nd[2], nd[3], id[0], id[1], id[2], id[3], m, Table{mn, mi}, out);
        std::printf("%%d", k);
        for (int r = 0; r < k; ++r) std::printf(" %%d %%d %%d %%d", out[r][0], out[r][1], out[r][2], out[r][3]);
        std::printf("\n");
    }
    return 0;
}
"""


def _run_rule_driver(tmp_path, nodes, ids, mask, mn, mi):
    src = tmp_path / "rule.cpp"
    src.write_text(RULE_DRIVER % HEADER)
    exe = tmp_path / "rule"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True, capture_output=True)
    lines = []
    for q in range(nodes.shape[0]):
        vals = list(nodes[q]) + list(ids[q]) + [mask[q]] + list(mn[q].ravel()) + list(mi[q].ravel())
        lines.append(" ".join(str(int(v)) for v in vals))
    r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    out = []
    for row in r.stdout.strip().split("\n"):
        v = [int(x) for x in row.split()]
        out.append(np.array(v[1:], dtype=np.int64).reshape(v[0], 4).tolist())
    return out


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_cuda_split_rule_matches_the_oracle(tmp_path):
    """The CUDA path's whole split rule (cem_split_subs, compiled here for the host)
    gives the oracle's sub-elements, in the oracle's order: for random elements with
    every side mask, and for the notch splits of three notched blocks."""
    from cem_inputs import kuhn_block
    from oracle import CEMOracle
    from split_cases import notch_cases, random_cases
    sets = [random_cases(2000, 21)]
    for k, w in enumerate([kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, traction=1.5e6),
                           kuhn_block(5, 4, 1, 0.025, 0.02, 0.005, notch_length=0.012, E_cov=0.2, seed=8),
                           kuhn_block(16, 8, 3, 0.08, 0.04, 0.015, notch_length=0.04)]):
        sets.append(notch_cases(CEMOracle.from_workload(w, split_enabled=False), 30 + k))
    for nodes, ids, mask, mn, mi, want in sets:
        got = _run_rule_driver(tmp_path, nodes, ids, mask, mn, mi)
        assert got == want
