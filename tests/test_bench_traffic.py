"""bench.py --record-traffic: DRAM bytes per launch from an ncu CSV capture,
recorded with each kernel's source hash, and used by the roofline only while
the source is unchanged (CPU only, synthetic CSV)."""
import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _write_csv(path, launches):
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HDR)
        for lid, name, rd, wr in launches:
            for metric, unit, val in (("dram__bytes_read.sum", "Gbyte", rd), ("dram__bytes_write.sum", "Mbyte", wr),
                                      ("gpu__time_duration.sum", "msecond", "1.5")):
                w.writerow([str(lid), "1", "python3", "host", name, "1", "7", "(256, 1, 1)", "(10, 1, 1)", "0",
                            "10.3", "Command line profiler metrics", metric, unit, val])


def test_record_traffic(tmp_path):
    launches = [
        (0, "void fastgb::(anonymous namespace)::k_sig_walk<(bool)1>(const unsigned short *, unsigned long)",
         "6.2", "3,000.5"),
        (1, "void fastgb::<unnamed>::k_pairs_grp<(int)2, unsigned int>(EnumArgs, unsigned int)", "17.0", "12,800"),
        (2, "void unnamed>::k_pairs_grp<(int)2, unsigned int>(EnumArgs, unsigned int)", "99", "99"),  # second launch
        (3, "void unnamed>::k_warp_vote<unsigned int>(VoteArgs, const T1 *)", "5.4", "2"),
        (4, "void unnamed>::k_scatter<unsigned int, 1, 0, 0>(const T1 *)", "1", "1"),  # not recorded
    ]
    src = tmp_path / "t.csv"
    out = tmp_path / "dt.json"
    _write_csv(src, launches)
    rec = bench.record_traffic(str(src), 1_000_000, "cmd", str(out))
    assert set(rec) == {"k_sig_walk", "k_pairs_grp<2>", "k_warp_vote"}
    assert rec["k_sig_walk"]["dram_read_bytes"] == 6.2e9
    assert rec["k_sig_walk"]["dram_write_bytes"] == 3000.5e6
    assert rec["k_pairs_grp<2>"]["dram_read_bytes"] == 17.0e9  # the first launch only
    assert abs(rec["k_warp_vote"]["bytes_per_unit"] - (5.4e9 + 2e6) / 1e6) < 1e-6
    on_disk = json.load(open(out))
    assert on_disk == json.loads(json.dumps(rec))
    for name, r in rec.items():
        assert r["source_sha256_16"] == bench._kernel_source_hash(r["source"]), name


def test_committed_traffic_matches_its_sources():
    # every committed record names a source file of this repository and the
    # hash format the roofline checks against
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    assert "k_sig_walk" in rec
    for name, r in rec.items():
        assert os.path.exists(os.path.join(ROOT, r["source"])), name
        assert len(r["source_sha256_16"]) == 16 and r["bytes_per_unit"] > 0
        assert r["unit"] == "fingerprint"
