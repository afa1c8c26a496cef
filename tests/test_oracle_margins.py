"""Conditioning of the FP64 parity runs, no GPU: how near each split decision of
the oracle lies to its switch point (Sec. 3, Eqs. 16-18).

The FP64 parity tests demand identical split records from two correct
implementations that round differently (the CUDA path's closed-form
eigen-projection against LAPACK, a factored force against the assembled
one; they agree on G to 1e-9 relative).  That bar is fair only if no decision
of those runs lies within that discrepancy of its switch point.  For every
FP64 parity workload with splitting, this runs the oracle over the same steps,
lists the candidates whose G lies within 1e-6 of Gc, and checks each margin
(CEMOracle.decision_margins) against the discrepancy the two sides can have
in that quantity.
"""
import numpy as np
import pytest

from cem_inputs import kuhn_block, plate_small
from oracle import CEMOracle

# smallest admissible margins: G, pattern and face choices against the 1e-9 agreement
# of G (a factor 10 above it); the stretch switch l / L - 1 against its rounding
# (about 1e-15 for these element sizes); the principal-stress gap so that an eigenvector
# perturbation of sigma's discrepancy / gap stays far below the G margins
FLOOR = {"G": 1e-8, "pattern": 1e-8, "face": 1e-8, "stretch": 1e-13, "eigen": 1e-4}


def _pulled_block():
    """The velocity-ramp workload of the GPU variant tests (jitter 0.1, seed 5)."""
    w = kuhn_block(20, 8, 2, 0.1, 0.04, 0.01, notch_length=0.05, traction=0.0, jitter=0.1, seed=5)
    y = w.X[:, 1]
    top = np.nonzero(np.isclose(y, y.max()))[0]
    bot = np.nonzero(np.isclose(y, 0.0))[0]
    dn = np.concatenate([bot, bot, bot, top])
    dc = np.concatenate([np.zeros(bot.size, int), np.ones(bot.size, int), np.full(bot.size, 2),
                         np.ones(top.size, int)])
    dv = np.concatenate([np.zeros(3 * bot.size), np.full(top.size, 2.0)])
    return w, dict(dirichlet=(dn, dc, dv, 5e-6))


def _hetero():
    return kuhn_block(13, 6, 3, 0.065, 0.03, 0.015, notch_length=0.03, jitter=0.15, E_cov=0.1, Gc_cov=0.2,
                      seed=3, traction=2e6), {}


CASES = {
    "block_20x8x2": (lambda: (plate_small(), {}), 2000),
    "jittered_heterogeneous": (_hetero, 450),
    "deactivate": (lambda: (plate_small(), dict(split_mode="deactivate")), 1200),
    "normal_traction": (lambda: (plate_small(), dict(g_variant="normal")), 1200),
    "velocity_ramp": (_pulled_block, 750),
}


@pytest.mark.parametrize("case", list(CASES))
def test_split_decisions_are_far_from_their_switch_points(case):
    make, steps = CASES[case]
    w, kw = make()
    o = CEMOracle.from_workload(w, **kw)
    o.margin_log = []
    o.step(steps)
    log = [(s, t, m) for s, t, m in o.margin_log if m is not None]
    assert o.energy()["n_split"] > 20 and len(log) > 100
    near = [(s, t, m["G"]) for s, t, m in log if m["G"] < 1e-6]
    print("\n%s: %d evaluations, %d splits; G within 1e-6 of Gc: %s" % (case, len(log), o.energy()["n_split"],
                                                                      near or "none"))
    for k, floor in FLOOR.items():
        worst = min(log, key=lambda r: r[2][k])
        print("  %-8s smallest margin %.3e (step %d, element %d)" % (k, worst[2][k], worst[0], worst[1]))
        assert worst[2][k] > floor, (k, worst)


def test_margins_see_a_decision_at_its_switch_point():
    # an element whose G is placed exactly on its Gc reports a zero G margin, and the
    # margins of a split element name its pattern and face gaps
    w = plate_small()
    o = CEMOracle.from_workload(w)
    o.step(200)
    t = next(t for t in o.candidates() if o.evaluate_candidate(t)[0] > 0.0)
    G = o.evaluate_candidate(t)[0]
    o.Gc_t[t] = G
    m = o.decision_margins(t)
    assert m["G"] == 0.0 and m["pattern"] == np.inf and m["face"] == np.inf
    o.Gc_t[t] = 0.5 * G
    m = o.decision_margins(t)
    assert abs(m["G"] - 1.0) < 1e-15 and 0.0 <= m["pattern"] <= 1.0
