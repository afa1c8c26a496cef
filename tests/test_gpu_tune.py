"""Autotuner of the step kernels' launch variants: every variant gives the same
bits, tuning leaves the simulation state unchanged, and the cache file is
written and reused."""
import itertools
import os

import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def CEM():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import CEM
    return CEM


BATCHES = {"strain": [1], "edge_stress": [2, 4, 8, 102, 104, 108, 200], "force": [1], "node_update": [2, 4, 8, 128]}


def _run(CEM, w, precision, variants=None, tune=None, steps=300):
    sim = CEM.from_workload(w, precision=precision)
    if tune is not None:
        sim.autotune(**tune)
    for k, (b, q) in (variants or {}).items():
        sim.tune_set(k, b, q)
    sim.step(steps)
    out = sim.field("u"), sim.field("v"), sim.crack_state()
    sim.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_variant_gives_identical_bits(CEM, precision):
    w = kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, seed=3, traction=2e6)
    u0, v0, c0 = _run(CEM, w, precision)
    assert len(c0) > len(w.notch_tet)
    for block in (128, 256, 512):
        for k, qs in BATCHES.items():
            for q in qs:
                u, v, c = _run(CEM, w, precision, variants={k: (block, q)})
                assert np.array_equal(u, u0) and np.array_equal(v, v0), (k, block, q)
                assert c == c0


def test_autotune_keeps_state_and_writes_cache(CEM, tmp_path):
    w = plate_small()
    path = str(tmp_path / "tune.txt")
    u0, v0, c0 = _run(CEM, w, "mixed")
    u1, v1, c1 = _run(CEM, w, "mixed", tune=dict(cache_path=path, reps=3, automatic=True))
    assert np.array_equal(u1, u0) and np.array_equal(v1, v0) and c1 == c0
    lines = open(path).read().strip().split("\n")
    assert len(lines) >= 4
    kernels = {l.split("\t")[1] for l in lines}
    assert kernels == {"strain", "edge_stress", "force", "node_update"}
    # a second context with the same sizes takes every choice from the cache (no timing)
    sim = CEM.from_workload(w, precision="mixed")
    t = sim.autotune(cache_path=path, reps=3, automatic=False)
    assert all(us == 0.0 for (_, _, us, _) in t.values())
    assert len(open(path).read().strip().split("\n")) == len(lines)


def test_tune_set_rejects_unknown_variants(CEM):
    from paper_2508_04076_gb300 import CEMError
    sim = CEM.from_workload(plate_small())
    with pytest.raises(CEMError):
        sim.tune_set("edge_stress", 64, 1)
    with pytest.raises(CEMError):
        sim.tune_set("node_update", 256, 3)
