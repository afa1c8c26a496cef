"""Thin ctypes binding of the CEM C ABI (include/cem.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory (its caching
allocator, installed as the library's allocator hook) and the stream.  There
is no CPU fallback: if the shared library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CEM_OK, CEM_EINVAL, CEM_ENOMEM, CEM_ECUDA = 0, -1, -2, -3
CEM_ECAPACITY, CEM_ENONFINITE, CEM_ETIMEOUT, CEM_ESTATE = -4, -5, -6, -7
CEM_FP64, CEM_MIXED = 0, 1
SPLIT_MODES = {"subdivide": 0, "deactivate": 1}
G_VARIANTS = {"principal": 0, "normal": 1}
FIELD = {"u": 0, "v": 1, "a": 2, "X": 3}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

EXPORTED = ["cem_mesh_create", "cem_set_material", "cem_step", "cem_set_step_batch", "cem_step_graph",
            "cem_step_persistent", "cem_energy", "cem_crack_state", "cem_get_field", "cem_info", "cem_energy_instance", "cem_adjoint", "cem_profile", "cem_profile_read",
            "cem_autotune", "cem_tune_get", "cem_tune_set", "cem_save", "cem_load", "cem_set_wait_limit",
            "cem_wait_probe", "cem_set_reorder", "cem_reorder_nodes", "cem_probe_fp64_fma", "cem_probe_split",
            "cem_probe_split_rule", "cem_node_energies_noalloc", "cem_destroy", "cem_last_error"]
TUNED = ["strain", "edge_stress", "force", "node_update"]
KERNELS = ["predict", "strain", "edge_stress", "force", "node_update", "front_G", "split"]


class MeshDesc(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64), ("n_tets", C.c_int64),
        ("X", C.POINTER(C.c_double)), ("tets", C.POINTER(C.c_int32)),
        ("n_tfaces", C.c_int64), ("tfaces", C.POINTER(C.c_int32)), ("tvec", C.POINTER(C.c_double)),
        ("n_notch", C.c_int64), ("notch_tet", C.POINTER(C.c_int32)), ("notch_side", C.POINTER(C.c_uint8)),
        ("precision", C.c_int32), ("dt", C.c_double), ("cfl_factor", C.c_double),
        ("split_enabled", C.c_int32), ("split_capacity", C.c_int64),
        ("stream", C.c_void_p), ("device", C.c_int32),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
        ("n_instances", C.c_int64), ("tet_instance", C.POINTER(C.c_int32)),
        ("split_mode", C.c_int32), ("g_variant", C.c_int32),
        ("n_dirichlet", C.c_int64), ("dir_node", C.POINTER(C.c_int32)), ("dir_comp", C.POINTER(C.c_uint8)),
        ("dir_v0", C.POINTER(C.c_double)), ("dir_t0", C.c_double),
        ("elem_type", C.c_int32), ("tface_nodes", C.c_int32),
    ]


class Energy(C.Structure):
    _fields_ = [("kinetic", C.c_double), ("strain", C.c_double), ("ext_work", C.c_double),
                ("dissipated", C.c_double), ("modified", C.c_double), ("step", C.c_int64),
                ("time", C.c_double), ("n_split", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tets", C.c_int64), ("n_active_tets", C.c_int64),
                ("n_edges", C.c_int64), ("n_candidates", C.c_int64), ("n_orig_edges", C.c_int64),
                ("dt", C.c_double), ("h_min", C.c_double), ("device_bytes", C.c_int64),
                ("n_reorder", C.c_int64), ("persistent_blocks", C.c_int64)]


_LIB = None


def load_library(build: bool = True):
    """Load libcem.so (building it first when asked and needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build:
        path = _build.build_library()
    if not os.path.exists(path):
        raise RuntimeError("libcem.so is not built; run paper_2508_04076_gb300.build.build_library()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.cem_mesh_create.argtypes = [C.POINTER(MeshDesc), C.POINTER(P)]
    lib.cem_set_material.argtypes = [P, C.c_double, C.c_double, C.POINTER(C.c_double), C.c_int64,
                                     C.POINTER(C.c_double), C.c_int64]
    lib.cem_step.argtypes = [P, C.c_int64]
    lib.cem_step_graph.argtypes = [P, C.c_int64]
    lib.cem_step_persistent.argtypes = [P, C.c_int64]
    lib.cem_set_step_batch.argtypes = [P, C.c_int64]
    lib.cem_energy.argtypes = [P, C.POINTER(Energy)]
    lib.cem_energy_instance.argtypes = [P, C.c_int64, C.POINTER(Energy)]
    lib.cem_adjoint.argtypes = [P, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.cem_crack_state.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int8),
                                    C.POINTER(C.c_uint8), C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int64]
    lib.cem_get_field.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int64)]
    lib.cem_info.argtypes = [P, C.POINTER(Info)]
    lib.cem_profile.argtypes = [P, C.c_int]
    lib.cem_profile_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_int64)]
    lib.cem_probe_fp64_fma.argtypes = [C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    lib.cem_probe_split.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_float), C.c_int64,
                                    C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_double)]
    I32 = C.POINTER(C.c_int32)
    lib.cem_probe_split_rule.argtypes = [C.c_int64, I32, I32, I32, I32, I32, I32, I32]
    lib.cem_autotune.argtypes = [P, C.c_char_p, C.c_int, C.c_int]
    lib.cem_tune_set.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.cem_save.argtypes = [P, C.c_char_p]
    lib.cem_set_wait_limit.argtypes = [P, C.c_int64]
    lib.cem_wait_probe.argtypes = [P]
    lib.cem_set_reorder.argtypes = [P, C.c_double]
    lib.cem_reorder_nodes.argtypes = [P]
    lib.cem_load.argtypes = [P, C.c_char_p]
    lib.cem_tune_get.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]
    lib.cem_node_energies_noalloc.argtypes = [P] * 5 + [C.c_int64, C.c_int64, P, P]
    lib.cem_destroy.argtypes = [P]
    lib.cem_last_error.argtypes = [P]
    lib.cem_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name != "cem_last_error":
            getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def probe_fp64_fma(device=0, stream=0) -> float:
    """Measured FP64 FMA throughput of the GPU in FLOP/s (FMA = 2 FLOP)."""
    lib = load_library()
    out = C.c_double()
    rc = lib.cem_probe_fp64_fma(int(device), C.c_void_p(int(stream)), C.byref(out))
    if rc != CEM_OK:
        raise CEMError(rc, "FP64 probe failed")
    return out.value


def probe_split(x, f):
    """(hi, lo, fd): the mixed node update's integer-only FP32 pair of each double x
    and float-to-double conversion of each float f, run on the current GPU."""
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float32)
    if x.shape != f.shape:
        raise ValueError("x and f must have the same shape")
    hi, lo, fd = np.empty(x.shape, np.float32), np.empty(x.shape, np.float32), np.empty(x.shape, np.float64)
    rc = lib.cem_probe_split(_ptr(x, C.c_double), _ptr(f, C.c_float), x.size, _ptr(hi, C.c_float),
                             _ptr(lo, C.c_float), _ptr(fd, C.c_double))
    if rc != CEM_OK:
        raise CEMError(rc, "split probe failed")
    return hi, lo, fd


def probe_split_rule(nodes, ids, mask, mnode, mid):
    """The split rule (sub-elements of a split element) run on the current GPU.

    nodes, ids: (n, 4) node indices of each element and their creation ids;
    mask: (n,) side masks; mnode, mid: (n, 4, 4), [q, x, y] = the new node on
    local edge x-y attached to x and its creation id.  Returns (subs, count):
    (n, 6, 4) sub-element nodes (rows past count[q] are -1) and (n,) counts."""
    lib = load_library()
    nodes = np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1, 4)
    n = nodes.shape[0]
    ids = np.ascontiguousarray(ids, dtype=np.int32).reshape(n, 4)
    mask = np.ascontiguousarray(mask, dtype=np.int32).reshape(n)
    mnode = np.ascontiguousarray(mnode, dtype=np.int32).reshape(n, 4, 4)
    mid = np.ascontiguousarray(mid, dtype=np.int32).reshape(n, 4, 4)
    subs, count = np.empty((n, 6, 4), np.int32), np.empty(n, np.int32)
    rc = lib.cem_probe_split_rule(n, _ptr(nodes, C.c_int32), _ptr(ids, C.c_int32), _ptr(mask, C.c_int32),
                                  _ptr(mnode, C.c_int32), _ptr(mid, C.c_int32), _ptr(subs, C.c_int32),
                                  _ptr(count, C.c_int32))
    if rc != CEM_OK:
        raise CEMError(rc, "split-rule probe failed")
    return subs, count


class CEMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("CEM error %d: %s" % (code, msg))
        self.code = code


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None and a.size else None


class CEM:
    """One simulation context on one GPU (C ABI: cem_mesh_create ... cem_destroy)."""

    def __init__(self, X, tets, tfaces=None, tvec=None, notch_tet=None, notch_side=None, *,
                 dt=0.0, cfl_factor=0.5, split_enabled=True, split_capacity=0, device=0,
                 stream=None, torch_allocator=True, precision="fp64", tet_instance=None,
                 split_mode="subdivide", g_variant="principal", dirichlet=None, elem="tet"):
        """dirichlet: None or (nodes, comps, v0, t0), prescribed velocity components
        v(t) = min(t / t0, 1) v0 (see cem_mesh_desc).  elem: "tet" (linear tetrahedra,
        traction triangles) or "hex" (trilinear hexahedra passed as `tets` with 8 nodes
        each, traction quadrilaterals; fixed topology)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the CEM library needs a CUDA GPU; no CPU fallback exists")
        self._lib = load_library()
        self._torch = torch
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = int(stream)
        if elem not in ("tet", "hex"):
            raise ValueError("elem must be 'tet' or 'hex'")
        npe, nf = (4, 3) if elem == "tet" else (8, 4)
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, npe)
        tfaces = np.ascontiguousarray(np.zeros((0, nf)) if tfaces is None else tfaces, dtype=np.int32).reshape(-1, nf)
        tvec = np.ascontiguousarray(np.zeros((0, 3)) if tvec is None else tvec, dtype=np.float64).reshape(-1, 3)
        notch_tet = np.ascontiguousarray([] if notch_tet is None else notch_tet, dtype=np.int32).ravel()
        notch_side = np.ascontiguousarray([] if notch_side is None else notch_side, dtype=np.uint8).ravel()
        inst = None if tet_instance is None else np.ascontiguousarray(tet_instance, dtype=np.int32).ravel()
        self.n_instances = 1 if inst is None else int(inst.max()) + 1
        if dirichlet is not None:
            dn, dc, dv, dt0 = dirichlet
            dn = np.ascontiguousarray(dn, dtype=np.int32).ravel()
            dc = np.ascontiguousarray(dc, dtype=np.uint8).ravel()
            dv = np.ascontiguousarray(dv, dtype=np.float64).ravel()
            if not (dn.size == dc.size == dv.size):
                raise ValueError("dirichlet nodes, components and velocities differ in length")
        else:
            dn = dc = dv = None
            dt0 = 0.0
        self._keep = (X, tets, tfaces, tvec, notch_tet, notch_side, inst, dn, dc, dv)
        d = MeshDesc()
        d.n_nodes, d.n_tets = X.shape[0], tets.shape[0]
        d.X, d.tets = _ptr(X, C.c_double), _ptr(tets, C.c_int32)
        d.n_tfaces, d.tfaces, d.tvec = tfaces.shape[0], _ptr(tfaces, C.c_int32), _ptr(tvec, C.c_double)
        d.elem_type, d.tface_nodes = (0, 3) if elem == "tet" else (1, 4)
        self.elem = elem
        d.n_notch, d.notch_tet, d.notch_side = notch_tet.size, _ptr(notch_tet, C.c_int32), _ptr(notch_side, C.c_uint8)
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        d.precision = CEM_FP64 if precision == "fp64" else CEM_MIXED
        self.precision = precision
        d.dt, d.cfl_factor = float(dt), float(cfl_factor)
        d.split_enabled, d.split_capacity = int(bool(split_enabled)), int(split_capacity)
        d.stream, d.device = self.stream, self.device
        if inst is not None and self.n_instances > 1:
            d.n_instances, d.tet_instance = self.n_instances, _ptr(inst, C.c_int32)
        if split_mode not in SPLIT_MODES or g_variant not in G_VARIANTS:
            raise ValueError("split_mode must be one of %s, g_variant one of %s" % (list(SPLIT_MODES), list(G_VARIANTS)))
        d.split_mode, d.g_variant = SPLIT_MODES[split_mode], G_VARIANTS[g_variant]
        if dn is not None:
            d.n_dirichlet, d.dir_node, d.dir_comp, d.dir_v0 = dn.size, _ptr(dn, C.c_int32), _ptr(dc, C.c_uint8), _ptr(dv, C.c_double)
            d.dir_t0 = float(dt0)
        if torch_allocator:
            dev = self.device

            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(strm or 0))
                except Exception:
                    return None

            def _free(ptr, strm, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
            d.alloc, d.free = self._alloc_cb, self._free_cb
        else:
            self._alloc_cb = self._free_cb = None
            d.alloc, d.free = ALLOC_FN(), FREE_FN()
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.cem_mesh_create(C.byref(d), C.byref(ctx))
        if rc != CEM_OK:
            raise CEMError(rc, self._lib.cem_last_error(None).decode())
        self._ctx = ctx

    @classmethod
    def from_hex_workload(cls, w, **kw):
        """Context for a cem_inputs.HexWorkload (fixed topology) with its material set."""
        kw.setdefault("split_enabled", False)
        sim = cls(w.X, w.hexes, w.tquads, w.tvec, None, None, elem="hex", **kw)
        sim.set_material(w.rho, w.nu, w.E, np.array([1.0]))
        return sim

    @classmethod
    def from_workload(cls, w, **kw):
        """Context for a cem_inputs.Workload with its material set."""
        kw.setdefault("tet_instance", getattr(w, "tet_instance", None))
        sim = cls(w.X, w.tets, w.tfaces, w.tvec, w.notch_tet, w.notch_side, **kw)
        sim.set_material(w.rho, w.nu, w.E, w.Gc)
        return sim

    def _check(self, rc):
        if rc != CEM_OK:
            raise CEMError(rc, self._lib.cem_last_error(self._ctx).decode())

    def set_material(self, rho, nu, E, Gc):
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        Gc = np.ascontiguousarray(np.atleast_1d(Gc), dtype=np.float64)
        if E.size > 1 and np.all(E == E[0]):
            E = E[:1].copy()
        if Gc.size > 1 and np.all(Gc == Gc[0]):
            Gc = Gc[:1].copy()
        self._check(self._lib.cem_set_material(self._ctx, float(rho), float(nu), _ptr(E, C.c_double), E.size,
                                               _ptr(Gc, C.c_double), Gc.size))

    def step(self, n=1):
        self._check(self._lib.cem_step(self._ctx, int(n)))

    def set_step_batch(self, max_steps=32):
        """Longest batch of steps launched before the host reads the split decision
        (cem_set_step_batch); 1 reads it after every step."""
        self._check(self._lib.cem_set_step_batch(self._ctx, int(max_steps)))

    def step_graph(self, n=1):
        """n steps as one captured CUDA graph (cem_step_graph): with crack-front elements
        the graph ends at the first step that splits and the rest runs as step() runs it;
        bit-identical to step(n)."""
        self._check(self._lib.cem_step_graph(self._ctx, int(n)))

    def step_persistent(self, n=1):
        """n fixed-topology steps in one persistent cooperative launch with bounded grid
        barriers (cem_step_persistent); bit-identical to step(n)."""
        self._check(self._lib.cem_step_persistent(self._ctx, int(n)))

    def energy(self) -> dict:
        e = Energy()
        self._check(self._lib.cem_energy(self._ctx, C.byref(e)))
        return {k: getattr(e, k) for k, _ in Energy._fields_}

    def energy_instance(self, i) -> dict:
        """Energies of specimen i of an ensemble."""
        e = Energy()
        self._check(self._lib.cem_energy_instance(self._ctx, int(i), C.byref(e)))
        return {k: getattr(e, k) for k, _ in Energy._fields_}

    def adjoint(self, n_steps, c_strain=1.0, w_u=None, checkpoint_every=0):
        """(J, dJ/dE per input element, dJ/dalpha) of n_steps steps from the current state."""
        n_tets = self._keep[1].shape[0]
        dE = np.zeros(n_tets, dtype=np.float64)
        J, da = C.c_double(), C.c_double()
        wu = None if w_u is None else np.ascontiguousarray(w_u, dtype=np.float64).reshape(-1, 3)
        self._check(self._lib.cem_adjoint(self._ctx, int(n_steps), int(checkpoint_every), float(c_strain),
                                          _ptr(wu, C.c_double) if wu is not None else None, C.byref(J),
                                          _ptr(dE, C.c_double), C.byref(da)))
        return J.value, dE, da.value

    def autotune(self, cache_path=None, reps=5, automatic=True):
        """Pick the fastest launch variant of each step kernel (results unchanged)."""
        path = None if cache_path is None else os.fsencode(cache_path)
        self._check(self._lib.cem_autotune(self._ctx, path, int(reps), int(bool(automatic))))
        return self.tuning()

    def tune_set(self, kernel, block, batch):
        """Pin one kernel's launch variant (kernel: one of TUNED)."""
        self._check(self._lib.cem_tune_set(self._ctx, TUNED.index(kernel), int(block), int(batch)))

    def tuning(self) -> dict:
        """{kernel: (block, batch, us, default_us)} of the current launch variants."""
        out = {}
        for k, name in enumerate(TUNED):
            b, q, us, du = C.c_int(), C.c_int(), C.c_double(), C.c_double()
            self._check(self._lib.cem_tune_get(self._ctx, k, C.byref(b), C.byref(q), C.byref(us), C.byref(du)))
            out[name] = (b.value, q.value, us.value, du.value)
        return out

    def save(self, path):
        """Write the dynamic state to a checkpoint file (cem_save)."""
        self._check(self._lib.cem_save(self._ctx, os.fsencode(path)))

    def load(self, path):
        """Resume from a checkpoint written by a context of the same mesh and material (cem_load)."""
        self._check(self._lib.cem_load(self._ctx, os.fsencode(path)))

    def set_wait_limit(self, spins=0):
        """Polls before a bounded device wait gives up (0: the default)."""
        self._check(self._lib.cem_set_wait_limit(self._ctx, int(spins)))

    def wait_probe(self):
        """Run one bounded wait on a flag nothing sets; raises CEMError(CEM_ETIMEOUT)."""
        self._check(self._lib.cem_wait_probe(self._ctx))

    def set_reorder(self, growth=0.25):
        """Renumber node storage once the node count grew by this fraction (0: never)."""
        self._check(self._lib.cem_set_reorder(self._ctx, float(growth)))

    def reorder_nodes(self):
        """Renumber node storage now (results are unchanged; node ids stay creation ids)."""
        self._check(self._lib.cem_reorder_nodes(self._ctx))

    def info(self) -> dict:
        i = Info()
        self._check(self._lib.cem_info(self._ctx, C.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def field(self, which="u") -> np.ndarray:
        n = C.c_int64()
        self._check(self._lib.cem_get_field(self._ctx, FIELD[which], None, 0, C.byref(n)))
        out = np.empty((n.value, 3), dtype=np.float64)
        self._check(self._lib.cem_get_field(self._ctx, FIELD[which], _ptr(out, C.c_double), out.size, C.byref(n)))
        return out

    def crack_state(self):
        """Split original elements sorted by (step, element): list of (tet, step, pattern, side, G)."""
        n = C.c_int64()
        self._check(self._lib.cem_crack_state(self._ctx, C.byref(n), None, None, None, None, None, 0))
        m = n.value
        tet = np.empty(m, np.int32)
        pat = np.empty(m, np.int8)
        side = np.empty(m, np.uint8)
        step = np.empty(m, np.int64)
        G = np.empty(m, np.float64)
        self._check(self._lib.cem_crack_state(self._ctx, C.byref(n), _ptr(tet, C.c_int32), _ptr(pat, C.c_int8),
                                              _ptr(side, C.c_uint8), _ptr(step, C.c_int64), _ptr(G, C.c_double), m))
        return [(int(tet[i]), int(step[i]), int(pat[i]), int(side[i]), float(G[i])) for i in range(m)]

    def profile(self, every=1):
        """Start (and clear) per-kernel CUDA-event timing on every `every`-th step; 0 / False stops."""
        self._check(self._lib.cem_profile(self._ctx, int(every)))

    def profile_read(self):
        """{kernel: (total_ms, launches)} and the total kernel launches since profile(True)."""
        n = len(KERNELS)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        tot = C.c_int64()
        self._check(self._lib.cem_profile_read(self._ctx, ms, cnt, n, C.byref(tot)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNELS)}, tot.value

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.cem_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
