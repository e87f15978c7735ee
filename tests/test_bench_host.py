"""Host-side logic of bench.py, CPU only: the whole-job time over ranks
(world size 2 on gloo), the rank environment, the clock summary and the
traffic record lookup."""
import os
import socket
import time

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    bench.barrier(world)
    slowest = bench.max_over_ranks(1.5 + rank, world)
    with open(os.path.join(out_dir, "rank%d" % rank), "w") as f:
        f.write(repr(slowest))
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert float((tmp_path / ("rank%d" % r)).read_text()) == 2.5


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_clock_summary_parses_samples():
    cs = bench.ClockSampler("0")
    now = time.time()
    cs.samples = [(now + 0.1 * k, [str(v), "2070", "700.5", "0x0", "Not Active", "Not Active", "Not Active",
                                   "Active" if k == 3 else "Not Active"]) for k, v in enumerate([2070, 2055, 2070, 1980])]
    s = cs.summary(now, now + 0.5)
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    assert cs.summary(now + 10, now + 11)["samples"] == 0


def test_recorded_traffic_requires_matching_kernel_sources(tmp_path, monkeypatch):
    f = tmp_path / "t.md"
    f.write_text("source_hash: %s\ndram_bytes_per_frame: 1.5e8\n" % bench.kernel_source_hash())
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic(32) == pytest.approx(4.8e9)
    f.write_text("source_hash: 0000\ndram_bytes_per_frame: 1.5e8\n")
    assert bench.recorded_traffic(32) is None


def test_edge_statistics_invariants():
    """The edge statistics of the bench line: four walks per edge fragment,
    every walk at most max_dist + 1 texels long, and only unfinished walks
    may reach that length."""
    import numpy as np
    import torch
    import bench
    rng = np.random.default_rng(3)
    depth = np.where(rng.random((64, 64)) < 0.3, np.float32(0.4), np.float32(1.0)).astype(np.float32)
    xyz = np.stack([rng.random(5000), rng.random(5000), np.full(5000, 0.9)]).astype(np.float32)
    host = [{"depth": torch.from_numpy(depth), "xyz": torch.from_numpy(xyz)}]
    e = bench.edge_statistics(host, per_frame=4000, max_dist=8)
    h = e["walk_length_histogram"]
    assert h["length"] == list(range(1, 10))
    assert e["sample_fragments"] == 4000
    n_edge = round(e["fraction"] * 4000)
    assert 0 < n_edge < 4000
    assert e["walks"] == 4 * n_edge == sum(h["end_found"]) + sum(h["no_end"])
    assert h["end_found"][-1] == 0 and e["capped_walks"] == h["no_end"][-1]


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference: rank 0 times the oracle on the host cores and prints
    one JSON line with the arm's keys; other ranks print nothing."""
    import json
    import rbsm_scenes as sc

    class Tiny:
        def __init__(self, seed):
            self.f = sc.config1(seed)

        def frame(self, k):
            return self.f

    monkeypatch.setattr(sc, "Config5", Tiny)
    args = bench.parse_args(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    bench.run_reference(args, 1, 2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
