"""Roofline accounting of bench.py (host arithmetic, no GPU): shares, the dominant
kernel, algorithmic bytes integrated window by window over a growing mesh, and the
FP64 ALU bound."""
import bench

UNITS = {"tets": "n_active_tets", "edges": "n_edges", "nodes": "n_nodes"}


def _prof(ms):
    p = {k: (ms.get(k, 0.0), 4 if k in ms else 0) for k in bench.KERNEL_UNITS}
    p["front_G"] = (0.2, 4)
    p["split"] = (0.0, 0)
    return p


def test_constant_mesh():
    counts = {"n_active_tets": 1000.0, "n_edges": 1250.0, "n_nodes": 210.0}
    ms = {"strain": 0.4, "edge_stress": 1.2, "force": 0.8, "node_update": 0.9}
    prof = _prof(ms)
    chunks = [(counts, {k: prof[k] for k in bench.KERNEL_UNITS})]
    kernels, roof = bench.roofline_accounting(chunks, prof, "mixed", 16.0, 50.0, 6000.0, 2070.0)
    fl, by = bench.kernel_costs(1000.0, 1250.0, 210.0, "mixed")
    assert roof["kernel"] == "edge_stress" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    per_launch_s = 1.2e-3 / 4
    assert roof["algorithmic_bytes_per_launch"] == by["edge_stress"] * 1250.0
    achieved = by["edge_stress"] * 1250.0 / per_launch_s / 1e9
    assert abs(roof["achieved"] - achieved) <= 1e-12 * achieved
    assert abs(roof["frac"] - achieved / 6000.0) <= 1e-12
    assert abs(roof["traffic"] - bench.DRAM_BYTES_PER_UNIT["mixed"]["edge_stress"] * 1250.0) <= 1e-6
    assert abs(kernels["edge_stress"]["share"] - 1.2 * 16.0 / 50.0) <= 1e-12
    assert abs(kernels["front_G"]["ms"] - 0.2 * 16.0) <= 1e-12
    for k in bench.KERNEL_UNITS:
        if k in ms:
            units = counts[UNITS[bench.KERNEL_UNITS[k]]]
            assert abs(kernels[k]["gbs"] - by[k] * units * 4 / (ms[k] * 1e-3) / 1e9) <= 1e-9 * kernels[k]["gbs"]


def test_growing_mesh_is_integrated_per_window():
    c1 = {"n_active_tets": 1000.0, "n_edges": 1200.0, "n_nodes": 200.0}
    c2 = {"n_active_tets": 4000.0, "n_edges": 9000.0, "n_nodes": 2000.0}
    w1 = {k: (0.1, 1) for k in bench.KERNEL_UNITS}
    w2 = {k: (0.3, 3) for k in bench.KERNEL_UNITS}
    w1["node_update"], w2["node_update"] = (0.5, 1), (3.0, 3)
    prof = {k: (w1[k][0] + w2[k][0], w1[k][1] + w2[k][1]) for k in bench.KERNEL_UNITS}
    prof["front_G"], prof["split"] = (0.0, 4), (0.0, 0)
    _, roof = bench.roofline_accounting([(c1, w1), (c2, w2)], prof, "mixed", 1.0, 10.0, 6000.0, 2070.0)
    _, b1 = bench.kernel_costs(1000.0, 1200.0, 200.0, "mixed")
    _, b2 = bench.kernel_costs(4000.0, 9000.0, 2000.0, "mixed")
    assert roof["kernel"] == "node_update"
    per_launch = (1 * b1["node_update"] * 200.0 + 3 * b2["node_update"] * 2000.0) / 4
    assert abs(roof["algorithmic_bytes_per_launch"] - per_launch) <= 1e-9 * per_launch
    assert abs(roof["units_per_launch"] - (200.0 + 3 * 2000.0) / 4) <= 1e-9
    # the mean of the end counts would misstate the bytes of a mesh that grows unevenly
    _, bm = bench.kernel_costs(2500.0, 5100.0, 1100.0, "mixed")
    assert abs(bm["node_update"] * 1100.0 - per_launch) > 1e-3 * per_launch


def test_fp64_path_is_alu_bound():
    counts = {"n_active_tets": 1000.0, "n_edges": 1250.0, "n_nodes": 210.0}
    ms = {"strain": 2.0, "edge_stress": 1.0, "force": 2.5, "node_update": 0.5}
    prof = _prof(ms)
    _, roof = bench.roofline_accounting([(counts, {k: prof[k] for k in bench.KERNEL_UNITS})], prof, "fp64", 1.0,
                                        20.0, 6000.0, 2000.0)
    fl, _ = bench.kernel_costs(1000.0, 1250.0, 210.0, "fp64")
    assert roof["kernel"] == "force" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["peak"] - 152 * 4 * 2000.0e6 / 1e12) <= 1e-12
    achieved = fl["force"] * 1000.0 / (2.5e-3 / 4) / 1e12
    assert abs(roof["achieved"] - achieved) <= 1e-12 * achieved
    assert roof["traffic"] is None
