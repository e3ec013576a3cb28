"""bench.py host logic (no GPU): the bytes model of the roofline and the
rule that measured DRAM traffic is used only while the ncu summary names the
current kernel sources."""
import bench


def test_bytes_model_per_unit():
    # x, u, tau read and written; photons: read x, u, tau, write x (and tau
    # with pairs); appended particle: its arrays plus the parent's weight
    assert bench.species_bytes(3, True) == (112, 88, 64)
    assert bench.species_bytes(2, True) == (96, 72, 56)
    assert bench.species_bytes(3, False) == (112, 80, 64)


def test_traffic_is_read_only_for_the_current_kernel_sources(tmp_path, monkeypatch):
    sid = bench.kernel_source_id()
    assert len(sid) == 12 and int(sid, 16) >= 0
    (tmp_path / "k_step_x.md").write_text(
        "# summary\n\n"
        f"traffic, mixed: read 1000 B, write 24 B per launch, kernel source {sid}\n"
        "traffic, fp64: read 2000 B, write 8 B per launch, kernel source 000000000000\n"
        f"traffic, fp32: read 300 B, write 100 B per launch, algorithmic 200 B per launch, "
        f"kernel source {sid}\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.measured_traffic("k_step_x.md", "mixed") == (1000, 24, None)
    assert bench.measured_traffic("k_step_x.md", "fp64") is None   # other sources
    assert bench.measured_traffic("k_step_x.md", "fp32") == (300, 100, 200)
    assert bench.measured_traffic("absent.md", "mixed") is None


def test_kernel_source_id_follows_the_step_sources_only(tmp_path, monkeypatch):
    # a copy of the sources: the id changes with a step source, not with
    # another unit of the library
    import shutil
    root = tmp_path / "r"
    for d in ("paper_1311_1107_gb300", "include"):
        shutil.copytree(bench.ROOT + "/" + d, root / d,
                        ignore=shutil.ignore_patterns("_build", "*.so", "__pycache__"))
    monkeypatch.setattr(bench, "ROOT", str(root))
    sid = bench.kernel_source_id()
    csrc = root / "paper_1311_1107_gb300" / "csrc"
    (csrc / "qp_pic.cu").write_text((csrc / "qp_pic.cu").read_text() + "// x\n")
    assert bench.kernel_source_id() == sid
    (csrc / "qp_step.cuh").write_text((csrc / "qp_step.cuh").read_text() + "// x\n")
    assert bench.kernel_source_id() != sid


def test_roofline_reports_traffic_and_fraction():
    res = {"lep_slots": 1000, "pho_slots": 0, "photons_added": 0, "pairs_added": 0,
           "kernel_ms": [1e-3, 0.0, 0.0], "launches": [1, 0, 0]}
    r = bench.roofline(res, 3, True, 100.0, "measured", (50, 10, None))
    assert r["achieved"] == 112.0 and r["frac"] == 1.12  # 112 kB in 1 us
    assert r["traffic"] == 60 and r["traffic_read_write"] == [50, 10]
    assert "traffic_scaled" not in r
    assert bench.roofline(res, 3, True, 100.0, "measured")["traffic"] is None
    # a capture of a smaller case (algorithmic 56 kB a launch): scaled by 2
    s = bench.roofline(res, 3, True, 100.0, "measured", (50_000, 10_000, 56_000))
    assert s["traffic_read_write"] == [100_000, 20_000] and s["traffic"] == 120_000
    assert "x2.000" in s["traffic_scaled"]


def test_roofline_counts_decayed_photons_as_their_tau_read_only():
    res = {"lep_slots": 1000, "pho_slots": 500, "dead_slots": 300, "photons_added": 0,
           "pairs_added": 0, "kernel_ms": [1e-3, 0.0, 0.0], "launches": [1, 0, 0]}
    r = bench.roofline(res, 3, True, 100.0, "measured")
    assert r["bytes_per_launch"] == 1000 * 112 + 500 * 88 + 300 * 8


def test_all_core_oracle_steps_the_same_particles_as_one_core():
    # the sample split over processes steps the same electrons (each with its
    # own random streams) as the single-process run of the same sample
    spec = ("plane", 0, None, None)
    w = bench.workload(*spec)
    slots1, _, n1 = bench.oracle_sample(w, 96, 3, 16)
    slots2, _, n2 = bench.oracle_all_cores(spec, 96, 3, 16, 2)
    assert n1 == n2 == 96 and slots1 == slots2


def test_fused_window_issue_roofline(tmp_path, monkeypatch):
    sid = bench.kernel_source_id()
    (tmp_path / "k_fused_x.md").write_text(
        f"instructions, mixed: 1000000 warp instructions per window, kernel source {sid}\n"
        "instructions, fp64: 5 warp instructions per window, kernel source 000000000000\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.measured_instructions("k_fused_x.md", "mixed") == 1_000_000
    assert bench.measured_instructions("k_fused_x.md", "fp64") is None
    # 152 SMs x 4 a cycle x 2070 MHz = 1258.56 G warp-instructions/s peak;
    # 1e6 instructions in a 1 ms window: 1 G/s achieved
    r = bench.issue_roofline(1_000_000, 2.0, 2, 152)
    assert r["bound"] == "alu" and r["peak"] == 1258.6
    assert r["achieved"] == 1.0 and r["frac"] == round(1.0 / 1258.56, 4)
    assert bench.issue_roofline(None, 2.0, 2, 152)["frac"] is None


def test_end_to_end_bytes_count_the_copies_made():
    # in: all seven rows of the live slots and a count per species; back:
    # six rows (no weights) of the slots live before the step, seven of the
    # appended ones, and the counts
    h2d, d2h = bench.e2e_bytes([10, 0, 5], [12, 1, 7], [7, 7, 7])
    assert h2d == (10 * 56 + 8) + 8 + (5 * 56 + 8)
    assert d2h == (10 * 48 + 2 * 56 + 8) + (1 * 56 + 8) + (5 * 48 + 2 * 56 + 8)
    assert bench.e2e_bytes([0, 0, 0], [0, 0, 0], [8, 8, 8]) == (24, 24)
