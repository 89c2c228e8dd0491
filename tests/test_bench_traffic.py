"""bench.py --record-traffic: DRAM bytes per unit of work from an ncu CSV
capture and the captured run's own JSON line (its counters), recorded with
each kernel's source hash, and used by the roofline only while the source is
unchanged (CPU only, synthetic CSV)."""
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
        (2, "void unnamed>::k_medium_grp<(int)2, unsigned int>(EnumArgs, const uint4 *)", "3", "1,000"),
        (3, "void unnamed>::k_medium_grp<(int)2, unsigned int>(EnumArgs, const uint4 *)", "1", "500"),
        (4, "void unnamed>::k_warp_vote<unsigned int>(VoteArgs, const T1 *)", "5.4", "2"),
        (5, "void unnamed>::k_scatter<unsigned int, 1, 0, 0>(const T1 *)", "1", "1"),  # not recorded
    ]
    src = tmp_path / "t.csv"
    out = tmp_path / "dt.json"
    line = tmp_path / "line.log"
    _write_csv(src, launches)
    counters = {"n_pairs_small": 2_000_000, "n_emissions": 2_500_000}
    line.write_text("noise\n" + json.dumps({"config": {"workload": "c1@1000000: ...", "N_per_station": 1_000_000},
                                            "counters": counters}) + "\n")
    rec = bench.record_traffic(str(src), str(line), "cmd", str(out))
    assert set(rec) == {"k_sig_walk", "k_pairs_grp", "k_medium_grp", "k_warp_vote"}
    assert rec["k_sig_walk"]["dram_read_bytes"] == 6.2e9 and rec["k_sig_walk"]["unit"] == "fingerprint"
    assert rec["k_sig_walk"]["dram_write_bytes"] == 3000.5e6
    assert abs(rec["k_sig_walk"]["bytes_per_unit"] - (6.2e9 + 3000.5e6) / 1e6) < 1e-6
    assert rec["k_pairs_grp"]["unit"] == "small-bucket pair"
    assert abs(rec["k_pairs_grp"]["bytes_per_unit"] - (17.0e9 + 12800e6) / 2e6) < 1e-6
    # both launches of the medium kernel, per medium-bucket pair (500,000 of them)
    assert abs(rec["k_medium_grp"]["bytes_per_unit"] - (4e9 + 1500e6) / 5e5) < 1e-6
    assert abs(rec["k_warp_vote"]["bytes_per_unit"] - (5.4e9 + 2e6) / 2.5e6) < 1e-6
    on_disk = json.load(open(out))
    assert on_disk == {"c1@1000000/1000000": json.loads(json.dumps(rec))}
    for name, r in rec.items():
        assert r["source_sha256_16"] == bench._kernel_source_hash(r["source"]), name
    # a second workload is kept beside the first; the 12-station line sums
    # its batches' units (two runs: warm-up and timed step)
    line2 = tmp_path / "line2.log"
    batches = {"2+1": {"n_pairs_small": 1_000_000, "n_emissions": 1_500_000, "windows": 3_000_000},
               "1": {"n_pairs_small": 1_000_000, "n_emissions": 1_000_000, "windows": 1_000_000}}
    line2.write_text(json.dumps({"config": {"workload": "c2: ...", "windows_per_step": 4_000_000},
                                 "counters_by_batch": batches}) + "\n")
    rec2 = bench.record_traffic(str(src), str(line2), "cmd", str(out), runs=2)
    assert abs(rec2["k_sig_walk"]["bytes_per_unit"] - (6.2e9 + 3000.5e6) / 8e6) < 1e-6
    assert abs(rec2["k_pairs_grp"]["bytes_per_unit"] - (17.0e9 + 12800e6) / 4e6) < 1e-6
    assert abs(rec2["k_medium_grp"]["bytes_per_unit"] - (4e9 + 1500e6) / 1e6) < 1e-6
    assert abs(rec2["k_pairs_grp"]["bytes_per_run"] - (17.0e9 + 12800e6) / 2) < 1e-3
    assert set(json.load(open(out))) == {"c1@1000000/1000000", "c2/4000000"}
    # a line whose batches do not add up to the step records bytes per search only
    batches.pop("1")
    line2.write_text(json.dumps({"config": {"workload": "c2: ...", "windows_per_step": 4_000_000},
                                 "counters_by_batch": batches}) + "\n")
    rec3 = bench.record_traffic(str(src), str(line2), "cmd", str(out), runs=2)
    assert rec3["k_pairs_grp"]["bytes_per_unit"] is None and rec3["k_pairs_grp"]["bytes_per_run"] > 0


def test_committed_traffic_matches_its_sources():
    # every committed record names a workload (name/windows), a source file
    # of this repository, a unit the roofline knows and the hash format it
    # checks against
    every = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    for key, rec in every.items():
        name, windows = key.split("/")
        assert name and int(windows) > 0
        for kernel, r in rec.items():
            assert os.path.exists(os.path.join(ROOT, r["source"])), kernel
            assert len(r["source_sha256_16"]) == 16 and r["bytes_per_run"] > 0
            assert r["unit"] in (None, "fingerprint", "small-bucket pair", "medium-bucket pair", "emission")
            assert (r["unit"] is None) == (r["bytes_per_unit"] is None)


def test_meter_keeps_batches_of_equal_length_apart():
    # batches of the same total length (7 months: 7, 6+1, 5+2, 4+3) each keep
    # their own counters, with their window count, in the line
    st = {k: 1.0 for k in ("ms_" + s for s in bench.STAGES)}
    st.update({k: 3 for k in bench.COUNTERS}, n_launches=5, n_fingerprints=7)
    import synth
    m = bench.Meter(synth.scaled("c2", 1000))
    m.on = True
    for key in ("7", "6+1", "5+2", "4+3"):
        m.add(18_144_000, dict(st, n_emissions=len(key)), key)
    assert set(m.last) == {"7", "6+1", "5+2", "4+3"}
    assert all(c["windows"] == 18_144_000 for c in m.last.values())
    assert [m.last[k]["n_emissions"] for k in ("7", "6+1", "5+2", "4+3")] == [1, 3, 3, 3]
    assert m.launches == 20


def test_walk_steps_matches_simulated_walks():
    # the expected walk length of k_sig_walk's bound against walks simulated
    # on uniformly drawn fingerprints: a random ranking of [0, D), a tile of
    # 32 fingerprints of K bits, the walk read 8 steps at a time until every
    # fingerprint is hit
    import numpy as np
    rng = np.random.default_rng(7)
    for D, K in ((512, 40), (2048, 100)):
        lens = []
        for _ in range(3000):
            rank = rng.permutation(D)
            pos = np.empty(D, np.int64)
            pos[rank] = np.arange(D)
            first = [pos[rng.choice(D, K, replace=False)].min() + 1 for _ in range(32)]
            lens.append(-(-max(first) // 8) * 8)
        want = float(np.mean(lens))
        got = bench.walk_steps(D, K)
        assert abs(got - want) < 4 * np.std(lens) / np.sqrt(len(lens)) + 0.05, (D, K, got, want)
    # more set bits, shorter walks; one fingerprint per tile, shorter still
    assert bench.walk_steps(8192, 800) < bench.walk_steps(8192, 400)
    assert bench.walk_steps(8192, 400, tile=1) < bench.walk_steps(8192, 400)


def test_walk_bound_counts_both_walks_of_min_max():
    import synth
    w = synth.scaled("c1", 1000)  # Min-Max, b = 100 tables of r = 4: 200 functions, 400 walks
    wb = bench.walk_bound(w, 10.0, 1_000_000)
    assert abs(wb["lookups_per_fingerprint"] - 400 * bench.walk_steps(w.D, w.K) / 32) < 1e-9
    assert abs(wb["achieved"] - 1e6 * wb["lookups_per_fingerprint"] / 0.01) < 1e-3 * wb["achieved"]
    assert wb["unit"] == "lookups/s" and 0 < wb["frac"] < 1
