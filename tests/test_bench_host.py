"""Host logic of the benchmark (CPU): the operating-point options, the kernel
names it reports, and the lookup of committed DRAM-traffic records."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_point_options_round_trip():
    from paper_2411_17229_gb300 import dade
    pt = bench.parse_point("nprobe=20,alpha=0.8,delta_d=64,tile=128,threads=128,schedule=2,seed_lists=2,flags=12", dade)
    kw = bench.point_kw(pt)
    assert kw == {"mode": 0, "tile": 128, "spec": 8, "threads": 128, "schedule": 2, "flags": 12, "seed_lists": 2,
                  "stage_dims": 0, "list_chunk": 0, "tc_min_rows": 0}
    assert pt["alpha"] == 0.8 and pt["nprobe"] == 20


def test_kernel_names_follow_the_schedule():
    c2 = {"mode": 0, "threads": 128, "delta_d": 64, "schedule": 2, "seed_lists": 2, "flags": 12}
    assert bench.scan_kernel_name(c2, 128).startswith("k_dade_fast<128, 8, 4>")
    c3 = dict(c2, threads=256, seed_lists=3, flags=28)
    assert "split" in bench.scan_kernel_name(c3, 960)
    c4 = {"mode": 0, "threads": 128, "delta_d": 32, "schedule": 0, "flags": 4}
    assert bench.scan_kernel_name(c4, 768) == "k_scan<DADE>"
    assert bench.scan_kernel_name({"mode": 1, "threads": 256}, 128) == "k_fd_fast<256, 8>"
    rounds = {"mode": 0, "threads": 128, "delta_d": 32, "schedule": 3, "flags": 4}
    assert bench.scan_kernel_name(rounds, 768).startswith("k_lm_g<2> (row rounds")
    assert "k_lm_tc<2>" in bench.scan_kernel_name(dict(rounds, flags=36), 768)
    assert "split" in bench.scan_kernel_name(dict(rounds, flags=20), 768)
    lead_tc = bench.scan_kernel_name(dict(rounds, flags=38), 768)     # lead prefilter replaces the TC one
    assert lead_tc.startswith("k_scan<DADE, lead>") and "split" in lead_tc
    assert "split" in bench.scan_kernel_name(dict(rounds, delta_d=48), 768)


def test_traffic_records_match_only_their_point_and_sources():
    with open(os.path.join(ROOT, "profiles", "scan_traffic.json")) as f:
        recs = json.load(f)
    assert recs, "no committed traffic record"
    for r in recs:
        assert set(r) >= {"scan_cu_sha256_16", "workload", "point", "dram_bytes_per_launch", "kernels", "command"}
        assert r["dram_bytes_per_launch"] == sum(k["dram_read"] + k["dram_write"] for k in r["kernels"].values())
        assert "--clock-control none" in r["command"]
    current = [r for r in recs if r["scan_cu_sha256_16"] == bench.scan_source_hash()]
    for r in current:
        assert bench.recorded_traffic(dict(r["point"]), r["workload"]) == r["dram_bytes_per_launch"]
        other = dict(r["point"], nprobe=r["point"]["nprobe"] + 1)
        assert bench.recorded_traffic(other, r["workload"]) is None


def test_alu_bound_where_lists_are_shared():
    c2 = {"mode": 0, "delta_d": 64, "schedule": 2, "flags": 12}
    assert bench.list_major_point(c2, 128)
    assert bench.list_major_point(dict(c2, delta_d=32), 256)
    assert not bench.list_major_point(dict(c2, flags=28), 960)          # split: query-major
    assert not bench.list_major_point(dict(c2, schedule=0), 128)        # tile schedule
    assert not bench.list_major_point(c2, 64)                           # D <= 112: split fallback
    assert bench.list_major_point(dict(c2, schedule=3, delta_d=32), 768)   # row rounds
    assert not bench.list_major_point(dict(c2, schedule=3, flags=20), 768)
    assert not bench.list_major_point(dict(c2, schedule=3, delta_d=32, flags=38), 768)   # lead: query-major
    assert bench.list_major_point(dict(c2, delta_d=32, flags=14), 768)   # seeded: lead leaves it list-major


def test_hnsw_point_choice():
    rows = [{"recall": 0.93, "ms": 1.0}, {"recall": 0.96, "ms": 3.0}, {"recall": 0.97, "ms": 2.5},
            {"recall": 0.99, "ms": 9.0}]
    assert bench.hnsw_pick(rows, 0.95) == rows[2]          # fastest at the target
    assert bench.hnsw_pick(rows[:1], 0.95) == rows[0]       # none reaches it: the best recall
    assert bench.HNSW_WORKLOAD in bench.synth.WORKLOADS
    assert all(ef >= 1 for ef in bench.HNSW_EFS) and list(bench.HNSW_EFS) == sorted(bench.HNSW_EFS)


def test_serving_runs_the_tuned_round_options():
    """The serving sweep hands the point's row-round options (first-round rows,
    work-item chunk, tensor-core window) to the server, so its batches run the
    launches the timed step runs; a tile point serves on the tile schedule."""
    from unittest import mock

    import numpy as np

    from paper_2411_17229_gb300 import dade
    made = []

    class FakeServer:
        def __init__(self, ix, **kw):
            made.append(kw)

        def replay(self, q, ks, nps, alpha, delta_d, arrivals):
            n = q.shape[0]
            return np.zeros((n, 100), np.int64), None, np.full(n, 1e-3), 1e-3

        def stats(self):
            return {"slots": 4, "batches": 1, "queries": 1, "max_inflight": 1}

        def close(self):
            pass

    ix = mock.Mock()
    ix.info.n_clusters, ix.info.d_pad = 8192, 256
    q = np.zeros((10, 256), np.float32)
    rounds = {"schedule": dade.SCHED_ROUNDS, "tile": 16, "threads": 256, "list_chunk": 1024, "tc_min_rows": 16384,
              "flags": dade.FLAG_TC_PREFILTER | dade.FLAG_LEAD, "alpha": 0.98, "delta_d": 64}
    tile = {"schedule": dade.SCHED_TILE, "tile": 128, "threads": 128, "flags": dade.FLAG_QUERY_ORDER}
    with mock.patch.object(dade, "Server", FakeServer):
        bench.serve_sweep(dade, ix, q, rounds, (2000,), 0.01)
        bench.serve_sweep(dade, ix, q, tile, (2000,), 0.01)
    assert made[0]["schedule"] == dade.SCHED_ROUNDS and made[0]["tile"] == 16
    assert made[0]["list_chunk"] == 1024 and made[0]["tc_min_rows"] == 16384
    assert made[0]["flags"] == dade.FLAG_TC_PREFILTER           # the lead prefilter is not a serving option
    assert made[1]["schedule"] == dade.SCHED_TILE and made[1]["list_chunk"] == 0 and made[1]["tc_min_rows"] == 0
