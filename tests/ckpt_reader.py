"""Reader of the library's checkpoint files (cem_save), for tests that check the
device topology: elements, element-edge maps, fan and incidence lists.

Layout (csrc/cem_io.cu): the tag "CEMCKPT3", int64 header fields, then every
saved array preceded by its int64 byte count, and a closing 64-bit hash.
Handles tetrahedral single-specimen contexts without prescribed velocities,
in FP64 or mixed precision.
"""
import collections

import numpy as np

HDR = ["ELEM", "PREC", "N0", "T0", "E0", "NC", "TC", "EC", "FANCAP", "INCCAP", "HASHCAP", "NINST", "SPLITMODE", "N",
       "T", "E", "NCAND", "NSPLITALL", "NSPLITRUN", "NACTIVE", "FANTOP", "INCTOP", "STEP", "DT_BITS", "RENUMBERED",
       "REORDER_N", "NREORDER"]
LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
MIXED = 1


def read(path):
    """(header dict, arrays dict) of a checkpoint."""
    b = open(path, "rb").read()
    assert b[:8] == b"CEMCKPT3", "not a checkpoint"
    H = dict(zip(HDR, (int(x) for x in np.frombuffer(b, np.int64, len(HDR), 8))))
    assert H["ELEM"] == 0 and H["NINST"] == 1, "tetrahedral single-specimen checkpoints only"
    pos, chunks = 8 + 8 * len(HDR), []
    while pos < len(b) - 8:
        nb = int(np.frombuffer(b, np.int64, 1, pos)[0])
        chunks.append(b[pos + 8:pos + 8 + nb])
        pos += 8 + nb
    it = iter(chunks)
    f64 = lambda: np.frombuffer(next(it), np.float64)  # noqa: E731
    f32 = lambda: np.frombuffer(next(it), np.float32)  # noqa: E731
    i32 = lambda: np.frombuffer(next(it), np.int32)  # noqa: E731
    u8 = lambda: np.frombuffer(next(it), np.uint8)  # noqa: E731
    mixed = H["PREC"] == MIXED
    S = {}
    for k in ("X", "u", "v", "a", "fext"):
        S[k] = np.stack([f64() for _ in range(3)], 1)
    S["mass"], S["minv"], S["inc_off"], S["inc_cnt"] = f64(), f64(), i32(), i32()
    if mixed:
        S["uhl"] = f32()
    S["conn"] = np.stack([i32() for _ in range(4)], 1)
    S["t2e"] = np.stack([i32() for _ in range(6)], 1)
    S["anc"], S["active"] = i32(), u8().astype(bool)
    S["Vg"] = np.stack([f64() for _ in range(9)], 1)
    if mixed:
        S["Vg32"] = np.stack([f32() for _ in range(9)], 1)
    S["vol"], S["lam"], S["mu"] = f64(), f64(), f64()
    S["fan_off"], S["fan_cnt"], S["cl"], S["cm"], S["sumV"] = i32(), i32(), f64(), f64(), f64()
    if mixed:
        S["cl32"], S["cm32"] = f32(), f32()
    S["fan_pool"], S["inc_pool"] = i32(), i32()
    S["Gc"], S["side"], S["split_step"], S["split_G"], S["ud_tet"], S["cand_flag"] = f64(), u8(), i32(), f64(), f64(), u8()
    S["cand_list"] = i32() if H["NCAND"] > 0 else np.zeros(0, np.int32)
    S["node_of_key"] = i32()
    S["hkeys"], S["hvals"], S["hfirst"] = np.frombuffer(next(it), np.uint64), i32(), i32()
    S["Ud"], S["ext"], S["oe_n0"], S["oe_n1"] = f64(), i32(), i32(), i32()
    return H, S


def topology_errors(H, S):
    """Inconsistencies of the device topology, as a list of strings (empty when sound):
    node and edge indices in range, one edge id per node pair, fans and incidence
    lists equal to what the active elements imply (ascending), positive volumes
    equal to the elements' geometry."""
    N, E = H["N"], H["E"]
    act = S["active"]
    conn, t2e = S["conn"][act], S["t2e"][act]
    ids = np.where(act)[0]
    err = []
    if conn.size and (conn.min() < 0 or conn.max() >= N):
        err.append("node index out of range")
        return err
    if t2e.size and (t2e.min() < 0 or t2e.max() >= E):
        err.append("edge index out of range")
        return err
    edge_of = {}
    for j, row, erow in zip(ids, conn, t2e):
        if len(set(row.tolist())) != 4:
            err.append("element %d repeats a node" % j)
        for l, (p, q) in enumerate(LOCAL_EDGES):
            key = (min(row[p], row[q]), max(row[p], row[q]))
            if edge_of.setdefault(key, erow[l]) != erow[l]:
                err.append("node pair %s has two edge ids" % (key,))
    if len(set(edge_of.values())) != len(edge_of):
        err.append("an edge id names two node pairs")
    fans = collections.defaultdict(list)
    inc = collections.defaultdict(list)
    for j, row, erow in zip(ids, conn, t2e):
        for l in range(6):
            fans[int(erow[l])].append(int(j))
        for l in range(4):
            inc[int(row[l])].append(4 * int(j) + l)
    for k in range(E):
        o, c = int(S["fan_off"][k]), int(S["fan_cnt"][k])
        if S["fan_pool"][o:o + c].tolist() != sorted(fans.get(k, [])):
            err.append("fan of edge %d" % k)
    for i in range(N):
        o, c = int(S["inc_off"][i]), int(S["inc_cnt"][i])
        if S["inc_pool"][o:o + c].tolist() != sorted(inc.get(i, [])):
            err.append("incidence list of node %d" % i)
    X = S["X"]
    d = X[conn[:, 1:]] - X[conn[:, :1]]
    V = np.einsum("ij,ij->i", d[:, 0], np.cross(d[:, 1], d[:, 2])) / 6.0
    if V.size and V.min() <= 0.0:
        err.append("non-positive volume")
    if V.size and np.abs(V - S["vol"][act]).max() > 1e-12 * np.abs(V).max():
        err.append("stored volumes differ from the geometry")
    return err


def element_sets(H, S):
    """Sorted list of the active elements' node sets in creation ids."""
    ext = S["ext"]
    return sorted(tuple(sorted(int(ext[v]) for v in row)) for row in S["conn"][S["active"]])


def chunks(raw):
    """(offset, bytes) of every saved array of a checkpoint's raw bytes, in file order."""
    pos, out = 8 + 8 * len(HDR), []
    while pos < len(raw) - 8:
        nb = int(np.frombuffer(raw, np.int64, 1, pos)[0])
        out.append((pos + 8, nb))
        pos += 8 + nb
    return out


def rehash(raw):
    """The raw bytes with their closing 64-bit FNV-1a hash (offset basis
    0xcbf29ce484222325, prime 0x100000001b3, as published) recomputed."""
    h = 0xCBF29CE484222325
    for b in bytes(raw[:-8]):
        h = ((h ^ b) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    out = bytearray(raw)
    out[-8:] = h.to_bytes(8, "little")
    return out
