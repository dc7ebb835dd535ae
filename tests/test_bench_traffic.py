"""bench.py's DRAM-traffic record (host logic, no GPU): the ratio of the DRAM bytes
ncu reports for the pass launches to the library's algorithmic bytes for the same
run, per launch, and the source hash that ties it to the kernel it was taken on."""
import json

import bench


def _csv(path, launches):
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, (rd, wr) in enumerate(launches):
        rows.append(f'"{i}","pass_rb_kernel","dram__bytes_read.sum","Mbyte","{rd}"')
        rows.append(f'"{i}","pass_rb_kernel","dram__bytes_write.sum","Gbyte","{wr}"')
        rows.append(f'"{i}","pass_rb_kernel","gpu__time_duration.sum","usecond","1.0"')
    path.write_text("==PROF== ncu log line\n" + "\n".join(rows) + "\n")


def test_traffic_ratio_per_launch(tmp_path):
    # two captured launches of 500 MB read + 0.5 GB written; the library traced three
    # launches of 1.5 GB algorithmic bytes in all: per launch 1.0 GB against 0.5 GB
    _csv(tmp_path / "dram.csv", [(500, 0.5), (500, 0.5)])
    line = {"config": {"workload": "brickwork20", "tile_qubits": 12},
            "trace_all": {"pass_launches": 3, "pass_algorithmic_bytes": 1.5e9}}
    (tmp_path / "trace.json").write_text("noise\n" + json.dumps(line) + "\n")
    out = bench.write_traffic(str(tmp_path / "dram.csv"), str(tmp_path / "trace.json"),
                              out_path=str(tmp_path / "t.json"))
    assert out["dram_read_bytes"] == 1e9 and out["dram_write_bytes"] == 1e9
    assert out["launches_captured"] == 2 and out["launches_traced"] == 3
    assert out["dram_bytes_per_algorithmic_byte"] == 2.0
    assert abs(out["ratio_over_totals"] - 2e9 / 1.5e9) < 1e-4
    assert out["source_sha"] == bench._kernel_sha()
    assert json.load(open(tmp_path / "t.json")) == out
