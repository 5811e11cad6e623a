"""Host logic of bench.py that needs no GPU: the DRAM-traffic record built
from an ncu CSV (per-kernel sums, unit scaling, per-cluster scaling to the
256-cluster launch, the kernel-source hash that invalidates it)."""
import csv

import bench


def _write_csv(path, rows):
    cols = ["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        f.write("==PROF== a line ncu prints before the table\n")
        w.writerow(cols)
        for r in rows:
            w.writerow(r)


def test_traffic_from_csv(tmp_path):
    """Two captures (one kernel each) summed per kernel, units scaled, memsets
    counted per wave, divided by the captured call's algorithmic bytes."""
    p1, p2 = tmp_path / "a.csv", tmp_path / "b.csv"
    _write_csv(p1, [
        ["0", "void cbfs::k_phase_a<4>(cbfs::Wave, int)", "dram__bytes_read.sum", "Mbyte", "100"],
        ["0", "void cbfs::k_phase_a<4>(cbfs::Wave, int)", "dram__bytes_write.sum", "Mbyte", "50"],
        ["2", "k_validate(long, const long *, ...)", "dram__bytes_read.sum", "Gbyte", "9"],  # not traversal
        ["3", "void cbfs::k_emit<4>(cbfs::Wave, const int *)", "gpu__time_duration.sum", "us", "5"],  # not bytes
    ])
    _write_csv(p2, [
        ["0", "void cbfs::k_phase_b<4>(cbfs::Wave, int)", "dram__bytes_read.sum", "Gbyte", "1.5"],
        ["0", "void cbfs::k_phase_b<4>(cbfs::Wave, int)", "dram__bytes_write.sum", "byte", "1,000"],
        ["1", "void cbfs::k_phase_b<4>(cbfs::Wave, int)", "dram__bytes_read.sum", "Mbyte", "2"],
    ])
    run = {"n": 1000, "d": 2, "clusters": 4, "A": 10_000_000, "V": 100_000, "tune": {"slots": 4}}
    out = bench.traffic_from_csv([str(p1), str(p2)], run, "test")["traversal"]
    kernels = 100e6 + 50e6 + 1.5e9 + 1000 + 2e6
    memsets = bench.memset_bytes_per_wave(1000, 4)
    alg = 13 * 10_000_000 + 41 * 100_000 + 4 * 1000 * 17
    assert out["kernel_dram_bytes"] == int(kernels) and out["memset_bytes"] == memsets
    assert abs(out["dram_bytes_per_alg_byte"] - (kernels + memsets) / alg) < 1e-12
    assert out["per_kernel_bytes"]["cbfs::k_phase_a<4>"] == int(150e6)
    assert out["launches_captured"]["cbfs::k_phase_b<4>"] == 2
    assert "k_validate" not in " ".join(out["per_kernel_bytes"])
    assert out["source_hash"] == bench.kernel_source_hash() and len(out["source_hash"]) == 16
    assert memsets == (16 * 4 + 4 + 4) * 1000 + 2 * 4 * 33 + 288 * 56


def test_summary_of_a_line_keeps_every_workload():
    line = {"value": 1000.0, "ms_per_step": 150.0,
            "roofline": {"avg_launch_ms": 140.0, "frac": 1.0, "arcs_per_s": 5e11, "physical_frac": 0.3},
            "e2e": {"value": 900.0},
            "one_cluster_per_launch": {"batched_speedup": 2.3},
            "query": {"p50_ms": 0.1, "p99_ms": 0.2, "kernel": {"frac": 0.8}},
            "serving": {"saturation_qps": 7e8, "offered": {"0.5x": {"p50_ms": 0.4, "p99_ms": 0.7},
                                                           "0.8x": {"p50_ms": 0.8, "p99_ms": 2.0}}},
            "next": {"road_grid": {"gteps": 160.0, "alg_frac": 0.2, "ms_all_clusters": 770.0, "arcs_per_s": 2e11},
                     "bfs_comparison": {"bit_level_gain": 28.0}},
            "configs": {"label_construction_s24": {"traversal_ms": 1200.0, "alg_frac": 0.5, "arcs_per_s": 3e11},
                        "single_cluster_s14": {"random_centres": {"ms_per_call_device": 0.05},
                                               "centres_deg_ge_63": {"ms_per_call_device": 0.08}}}}
    s = bench.summary_of(line)
    assert s["garcs_per_s"] == 500.0 and s["physical_frac"] == 0.3
    assert s["batched_speedup_vs_one_cluster_per_launch"] == 2.3
    assert s["serving_0.8x_p50_p99_ms"] == [0.8, 2.0]
    assert s["road_grid_4096"]["alg_frac"] == 0.2 and s["labels_s24_1024"]["garcs_per_s"] == 300.0
    assert s["single_s14_ms"]["centres_deg_ge_63"] == 0.08 and s["bit_level_gain"] == 28.0
    # missing sections (a run with --no-next) leave their keys out or None
    short = {k: line[k] for k in ("value", "ms_per_step", "roofline")}
    s2 = bench.summary_of(short)
    assert s2["serving_0.5x_p50_p99_ms"] == [None, None] and "road_grid_4096" not in s2
    import json
    assert len(json.dumps(s)) < 1200


def test_lockstep_rounds_counts_idle_slot_rounds():
    # sizes 5, 3, 9, 1 in waves of 2 by size: (9, 5) and (3, 1)
    ks = [5, 3, 9, 1]
    rounds = [4, 6, 8, 2]
    out = bench.lockstep_rounds(ks, rounds, 2)
    # 5 + 3 + 9 + 1 bits pack into one word: one wave of one word, 8 rounds
    assert out["words"] == 1 and out["waves"] == 1 and out["wave_rounds"] == 8
    assert out["cluster_rounds"] == 20 and out["busy_slot_round_share"] == 1.0
    # 64-source clusters take a word each: equal sizes keep call order, waves (0, 1) and (2, 3)
    big = [64] * 4
    out = bench.lockstep_rounds(big, rounds, 2)
    assert out["words"] == 4 and out["waves"] == 2 and out["wave_rounds"] == 6 + 8
    assert out["busy_slot_round_share"] == round(20 / (2 * 6 + 2 * 8), 4)


def test_pack_words_best_fit_largest_first():
    """Sizes 40, 30, 20, 10, 5, 64: 64 alone; 40 + 20 (best fit for 20: the
    word with 24 free) ; 30 + 10 + 5 ... and at most 31 clusters to a word."""
    words = bench.pack_words([40, 30, 20, 10, 5, 64])
    sizes = sorted(sorted([40, 30, 20, 10, 5, 64][c] for c in w) for w in words)
    assert sizes == [[5, 10, 30], [20, 40], [64]]
    ones = bench.pack_words([1] * 70)
    assert [len(w) for w in ones] == [31, 31, 8]
    assert bench.pack_words([64, 64]) == [[0], [1]]


def test_traffic_of_packed_waves_counts_waves_from_seed_launches(tmp_path):
    """A call whose waves write their outputs from round records (k_flush)
    and hold more clusters than slots: waves = k_seed launches, no Delta-row
    memsets."""
    p = tmp_path / "c.csv"
    _write_csv(p, [
        ["0", "cbfs::k_seed(cbfs::Wave, const unsigned long *, int)", "dram__bytes_read.sum", "byte", "100"],
        ["1", "cbfs::k_seed(cbfs::Wave, const unsigned long *, int)", "dram__bytes_read.sum", "byte", "100"],
        ["2", "void cbfs::k_flush_packed<4>(cbfs::Wave, const int *, int, int, int)", "dram__bytes_write.sum",
         "Mbyte", "7"],
    ])
    run = {"n": 1000, "d": 2, "clusters": 24, "A": 10_000_000, "V": 100_000, "tune": {"slots": 4}}
    out = bench.traffic_from_csv([str(p)], run, "test")["traversal"]
    assert out["waves"] == 2
    assert out["memset_bytes"] == 2 * bench.memset_bytes_per_wave(1000, 4, rows=False)
    assert out["memset_bytes"] == 2 * ((16 * 4 + 4) * 1000 + 2 * 4 * 33 + 288 * 56)
    assert out["per_kernel_bytes"]["cbfs::k_flush_packed<4>"] == int(7e6)


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2410_17226_gb300" / "csrc"
    csrc.mkdir(parents=True)
    f = csrc / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f.write_text('__global__ void k(int* x) { x[0] = 1; }\nconst char* s = "a // b";\n')
    h0 = bench.kernel_source_hash()
    f.write_text('// a kernel\n__global__ void k(int* x) {  /* one */\n  x[0] = 1;  // store\n}\n'
                 'const char* s = "a // b";\n')
    assert bench.kernel_source_hash() == h0
    f.write_text('__global__ void k(int* x) { x[0] = 2; }\nconst char* s = "a // b";\n')
    assert bench.kernel_source_hash() != h0
    f.write_text('__global__ void k(int* x) { x[0] = 1; }\nconst char* s = "a b";\n')
    assert bench.kernel_source_hash() != h0
