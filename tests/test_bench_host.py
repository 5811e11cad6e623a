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
    p = tmp_path / "t.csv"
    _write_csv(p, [
        ["0", "void cbfs::k_phase_a<4>(cbfs::Wave, int)", "dram__bytes_read.sum", "Mbyte", "100"],
        ["0", "void cbfs::k_phase_a<4>(cbfs::Wave, int)", "dram__bytes_write.sum", "Mbyte", "50"],
        ["1", "void cbfs::k_phase_b<4>(cbfs::Wave, int)", "dram__bytes_read.sum", "Gbyte", "1.5"],
        ["1", "void cbfs::k_phase_b<4>(cbfs::Wave, int)", "dram__bytes_write.sum", "byte", "1,000"],
        ["2", "k_validate(long, const long *, ...)", "dram__bytes_read.sum", "Gbyte", "9"],  # not traversal
        ["3", "void cbfs::k_emit<4>(cbfs::Wave, const int *)", "gpu__time_duration.sum", "us", "5"],  # not bytes
    ])
    out = bench.traffic_from_csv(str(p), 2, "test")["traversal"]
    total = 100e6 + 50e6 + 1.5e9 + 1000
    assert out["per_cluster_bytes"] == int(total / 2)
    assert out["dram_bytes_per_launch"] == int(total / 2 * 256)
    assert out["per_kernel_bytes"]["cbfs::k_phase_a<4>"] == int(150e6)
    assert "k_validate" not in " ".join(out["per_kernel_bytes"])
    assert out["source_hash"] == bench.kernel_source_hash() and len(out["source_hash"]) == 16
