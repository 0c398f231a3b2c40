"""Host-side check of bench.py's reference arm (no GPU needed): it times the
FP64 oracle on a bounded sample of the benchmark workload and prints one JSON
line with the fields the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    """The reference arm's line, on the SBM workload (the oracle finishes it in
    seconds; the 1M-node default differs only in the workload it times)."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "sbm2k", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("G-REST updates/s, SBM n=2,000")
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and 1 <= d["steps"] <= 2 and d["config"]["steps_requested"] == 2
    assert d["value"] > 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert "no scaling" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("SBM stream n=2,000")


def test_default_workload_is_the_1m_stream():
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS["cl1m"]
    assert w["metric"].startswith("G-REST updates/s at n=1M,k=32")
    assert bench.workload_desc(w).startswith("Chung-Lu power-law stream n=1,000,000 gamma=2.3 mean_degree=32 adjacency")
    assert (w["k"], w["L"], w["P"], w["op"]) == (32, 100, 100, 0)
    assert w["precisions"] == ("fp64", "mixed", "mixed_fast")


def test_capacity_covers_the_driver_run():
    """--steps 20 --warmup 5: every tracker applies W + K batches of +0.5%
    nodes (the end-to-end leg replays the same ones on a fresh tracker).  The
    contexts are created with room for all of them, so no growth (and no
    device-wide synchronizing free) falls inside a timed region."""
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS["cl1m"]
    nb = bench.batches_needed(20, 5)
    assert nb == 25
    g, batches = bench.make_workload(w, nb, w["seed"], n=20_000)
    assert len(batches) == nb
    n_final = g.n + sum(int(b.n_new) for b in batches)
    assert n_final > 1.1 * g.n
    cap = bench.stream_node_capacity(g.n, batches)
    assert cap >= n_final
    # every prefix fits too
    run = g.n
    for b in batches:
        run += int(b.n_new)
        assert run <= cap


def _replica_worker(rank, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    t_local = [1.5, 2.5][rank]
    t, rate = bench.replica_rate(t_local, 10, 2, device="cpu")
    m = bench.max_over_ranks(float(rank), 2, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate, "m": m}, f)


def test_replica_rate_over_two_gloo_ranks(tmp_path):
    """The N > 1 timing rule on two CPU ranks (gloo): every rank gets the
    slowest rank's time, and the whole-job rate counts both ranks' updates
    over that time."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_replica_worker, args=(port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["t"] == 2.5 and d["rate"] == 2 * 10 / 2.5 and d["m"] == 1.0


def test_reference_arm_other_ranks_exit_quietly():
    """Under a multi-rank launch only rank 0 runs the oracle and prints; the
    other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.strip().startswith("{")]


def test_roofline_traffic_per_kind_and_class(tmp_path, monkeypatch):
    """Traffic from an ncu summary: scaled by the node count, dropped for a
    kind whose sources changed since the capture, and combined into a class
    figure only when every launch of the class is of a kind with a figure."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    h = {k: bench.source_hash(v) for k, v in bench.KIND_SOURCES.items()}
    prof = tmp_path / "traffic.md"
    prof.write_text("\n".join([
        "| kind | launches per step | DRAM bytes per launch | mean node ids | sources hash |",
        "|---|---|---|---|---|",
        f"| `gram_tc` | 6 | 1000000 | 500000 | `{h['gram_tc']}` |",
        f"| `gram_narrow` | 7 | 200000 | 500000 | `{h['gram_narrow']}` |",
        f"| `gram_cuda` | 1 | 300000 | 500000 | `{h['gram_cuda']}` |",
        "| `gemm_tc` | 13 | 900000 | 500000 | `0123456789abcdef` |",  # stale: sources changed
    ]) + "\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    ms = np.array([7.0, 9.0, 7.0, 7.5, 1.0])
    work = np.full(5, 1e9)
    byts = np.full(5, 5e9)
    launches = np.array([5.0, 14.0, 16.0, 8.0, 1.0])
    kms = np.array([5.0, 2.0, 4.6, 1.9, 2.5, 4.5, 1.8, 0.0, 7.5, 1.0])
    kn = np.array([4.0, 1.0, 6.0, 7.0, 1.0, 13.0, 1.0, 0.0, 8.0, 1.0])
    r = bench.roofline(ms, work, byts, launches, (kms, np.full(10, 1e9), np.full(10, 1e9), kn), 1_000_000, "mixed")
    assert r["kernel_class"] == "gram"
    k = r["kernels"]
    assert k["gram_tc"]["traffic"] == 2_000_000 and k["gram_narrow"]["traffic"] == 400_000
    assert k["gemm_tc"]["traffic"] is None and k["spmm_f32"]["traffic"] is None
    assert k["gram_cuda"]["bound"] == "alu" and k["gram_tc"]["bound"] == "hbm"
    # the Gram class: 6 + 7 + 1 = 14 launches, all with a figure
    assert r["traffic"] == (6 * 2_000_000 + 7 * 400_000 + 1 * 600_000) / 14
    assert r["classes"]["gemm"]["traffic"] is None  # gemm_tc's figure is stale


def test_kind_sources_exist_and_profile_parses():
    """Every source file a traffic figure is tied to exists (a renamed file
    would silently drop the figure), and the committed ncu summary parses
    into one positive figure per kernel kind it lists."""
    sys.path.insert(0, ROOT)
    import bench
    for kind, files in bench.KIND_SOURCES.items():
        assert bench.source_hash(files) is not None, kind
    text = open(bench.TRAFFIC_PROFILE).read()
    rows = [l for l in text.splitlines() if l.startswith("| `") and l.count("|") == 6]
    assert {r.split("`")[1] for r in rows} == set(bench.KIND_SOURCES)
    for r in rows:
        cells = [c.strip() for c in r.strip("|").split("|")]
        assert float(cells[1]) > 0 and float(cells[2]) > 0 and float(cells[3]) > 0
