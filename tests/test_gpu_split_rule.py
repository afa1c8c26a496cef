"""The split rule of Sec. 3 run by the device code (cem_probe_split_rule) against
the oracle: the sub-elements of random elements with every side mask and of the
notch splits of three notched blocks, with storage indices drawn apart from
creation ids.  The division of each remaining prism into three tetrahedra must
cut every quadrilateral face through its smallest creation id, as the oracle's
does."""
import pytest

from split_cases import notch_cases, random_cases

pytestmark = pytest.mark.gpu


def test_device_split_rule_matches_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from cem_inputs import kuhn_block
    from oracle import CEMOracle
    from paper_2508_04076_gb300 import probe_split_rule
    sets = [random_cases(4000, 22)]
    for k, w in enumerate([kuhn_block(10, 4, 1, 0.05, 0.02, 0.005, notch_length=0.025, traction=1.5e6),
                           kuhn_block(5, 4, 1, 0.025, 0.02, 0.005, notch_length=0.012, E_cov=0.2, seed=8),
                           kuhn_block(16, 8, 3, 0.08, 0.04, 0.015, notch_length=0.04)]):
        sets.append(notch_cases(CEMOracle.from_workload(w, split_enabled=False), 40 + k))
    for nodes, ids, mask, mn, mi, want in sets:
        subs, count = probe_split_rule(nodes, ids, mask, mn, mi)
        got = [subs[q, : count[q]].tolist() for q in range(len(want))]
        assert got == want
