"""Roofline accounting of bench.py (host arithmetic, no GPU): the survey's
algorithmic bytes per element-step, their split over the kernels, shares, the
dominant kernel, window-by-window integration over a growing mesh, and the
FP64 ALU bound."""
import bench

UNITS = {"tets": "n_active_tets", "edges": "n_edges", "nodes": "n_nodes"}


def _prof(ms):
    p = {k: (ms.get(k, 0.0), 4 if k in ms else 0) for k in bench.KERNEL_UNITS}
    p["front_G"] = (0.2, 4)
    p["split"] = (0.0, 0)
    return p


def test_algorithmic_bytes_of_the_large_block():
    """The survey's section 8(d) figures for the 320x128x32 block: about 165 B per
    element-step in FP64 and about 139 B mixed; the kernels' shares sum to them."""
    T, E, N = 7864320.0, 9341408.0, 1366497.0
    assert abs(bench.b_alg_per_tet_step(T, E, N, "fp64") - 165.2) < 0.1
    assert abs(bench.b_alg_per_tet_step(T, E, N, "mixed") - 138.3) < 0.1
    for prec in ("fp64", "mixed"):
        _, alg, _ = bench.kernel_costs(T, E, N, prec)
        per = {"tets": 1.0, "edges": E / T, "nodes": N / T}
        tot = sum(alg[k] * per[bench.KERNEL_UNITS[k]] for k in bench.KERNEL_UNITS)
        assert abs(tot - bench.b_alg_per_tet_step(T, E, N, prec)) < 1e-9


def test_constant_mesh():
    counts = {"n_active_tets": 1000.0, "n_edges": 1250.0, "n_nodes": 210.0}
    ms = {"strain": 0.4, "edge_stress": 1.2, "force": 0.8, "node_update": 0.9}
    prof = _prof(ms)
    chunks = [(counts, 64, {k: prof[k] for k in bench.KERNEL_UNITS})]
    kernels, roof = bench.roofline_accounting(chunks, prof, "mixed", 16.0, 50.0, 6000.0, 1.2e12)
    fl, alg, mv = bench.kernel_costs(1000.0, 1250.0, 210.0, "mixed")
    assert roof["kernel"] == "edge_stress" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    per_launch_s = 1.2e-3 / 4
    assert roof["algorithmic_bytes_per_launch"] == alg["edge_stress"] * 1250.0
    assert roof["moved_bytes_per_launch"] == mv["edge_stress"] * 1250.0
    achieved = alg["edge_stress"] * 1250.0 / per_launch_s / 1e9
    assert abs(roof["achieved"] - achieved) <= 1e-12 * achieved
    assert abs(roof["frac"] - achieved / 6000.0) <= 1e-12
    assert abs(roof["traffic"] - bench.DRAM_BYTES_PER_UNIT["mixed"]["edge_stress"] * 1250.0) <= 1e-6
    assert abs(kernels["edge_stress"]["share"] - 1.2 * 16.0 / 50.0) <= 1e-12
    assert abs(kernels["front_G"]["ms"] - 0.2 * 16.0) <= 1e-12
    for k in bench.KERNEL_UNITS:
        if k in ms:
            units = counts[UNITS[bench.KERNEL_UNITS[k]]]
            assert abs(kernels[k]["alg_gbs"] - alg[k] * units * 4 / (ms[k] * 1e-3) / 1e9) <= 1e-9 * (
                kernels[k]["alg_gbs"] + 1e-30)
    ws = roof["whole_step"]
    b = bench.b_alg_per_tet_step(1000.0, 1250.0, 210.0, "mixed")
    assert abs(ws["alg_gbs"] - b * 1000.0 * 64 / 50e-3 / 1e9) <= 1e-9 * ws["alg_gbs"]
    assert abs(ws["hbm_frac"] - ws["alg_gbs"] / 6000.0) <= 1e-12


def test_growing_mesh_is_integrated_per_window():
    c1 = {"n_active_tets": 1000.0, "n_edges": 1200.0, "n_nodes": 200.0}
    c2 = {"n_active_tets": 4000.0, "n_edges": 9000.0, "n_nodes": 2000.0}
    w1 = {k: (0.1, 1) for k in bench.KERNEL_UNITS}
    w2 = {k: (0.3, 3) for k in bench.KERNEL_UNITS}
    w1["node_update"], w2["node_update"] = (0.5, 1), (3.0, 3)
    prof = {k: (w1[k][0] + w2[k][0], w1[k][1] + w2[k][1]) for k in bench.KERNEL_UNITS}
    prof["front_G"], prof["split"] = (0.0, 4), (0.0, 0)
    _, roof = bench.roofline_accounting([(c1, 16, w1), (c2, 48, w2)], prof, "mixed", 1.0, 10.0, 6000.0, 1.2e12)
    _, a1, _ = bench.kernel_costs(1000.0, 1200.0, 200.0, "mixed")
    _, a2, _ = bench.kernel_costs(4000.0, 9000.0, 2000.0, "mixed")
    assert roof["kernel"] == "node_update"
    per_launch = (1 * a1["node_update"] * 200.0 + 3 * a2["node_update"] * 2000.0) / 4
    assert abs(roof["algorithmic_bytes_per_launch"] - per_launch) <= 1e-9 * per_launch
    assert abs(roof["units_per_launch"] - (200.0 + 3 * 2000.0) / 4) <= 1e-9
    # the mean of the end counts would misstate the bytes of a mesh that grows unevenly
    _, am, _ = bench.kernel_costs(2500.0, 5100.0, 1100.0, "mixed")
    assert abs(am["node_update"] * 1100.0 - per_launch) > 1e-3 * per_launch
    # the whole step weights each window by its element-steps
    ws = roof["whole_step"]
    want = (bench.b_alg_per_tet_step(1000.0, 1200.0, 200.0, "mixed") * 1000.0 * 16
            + bench.b_alg_per_tet_step(4000.0, 9000.0, 2000.0, "mixed") * 4000.0 * 48) / (1000.0 * 16 + 4000.0 * 48)
    assert abs(ws["b_alg_per_element_step"] - want) <= 1e-9 * want
    assert abs(ws["active_element_steps_per_s"] - (1000.0 * 16 + 4000.0 * 48) / 10e-3) <= 1e-6


def test_fp64_path_is_alu_bound():
    counts = {"n_active_tets": 1000.0, "n_edges": 1250.0, "n_nodes": 210.0}
    ms = {"strain": 2.0, "edge_stress": 1.0, "force": 2.5, "node_update": 0.5}
    prof = _prof(ms)
    _, roof = bench.roofline_accounting([(counts, 4, {k: prof[k] for k in bench.KERNEL_UNITS})], prof, "fp64", 1.0,
                                        20.0, 6000.0, 1.25e12)
    fl, _, _ = bench.kernel_costs(1000.0, 1250.0, 210.0, "fp64")
    assert roof["kernel"] == "force" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["peak"] - 1.25) <= 1e-12
    achieved = fl["force"] * 1000.0 / (2.5e-3 / 4) / 1e12
    assert abs(roof["achieved"] - achieved) <= 1e-12 * achieved
    ws = roof["whole_step"]
    assert abs(ws["fp64_tflops"] - bench.flops_per_tet_step(1000.0, 1250.0, 210.0) * 1000.0 * 4 / 20e-3 / 1e12) \
        <= 1e-12 * ws["fp64_tflops"]


def test_hbm_peak_fallback_is_stated():
    assert bench._hbm_peak({"hbm_gbs": 6651.4}) == (6651.4, "of measured (MEASURED_PEAKS.json hbm_gbs)")
    v, src = bench._hbm_peak({})
    assert v == 6800.0 and src.startswith("of fallback")


def test_failing_leg_is_recorded():
    def boom():
        raise ValueError("x")
    assert bench._leg("ensemble", boom) == {"error": "ensemble: ValueError('x')"}
    assert bench._leg("ok", lambda: {"a": 1}) == {"a": 1}
