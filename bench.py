#!/usr/bin/env python3
"""G-REST update throughput on an evolving power-law graph (one JSON line).

Default workload (synthetic, seeded): Chung-Lu power-law graph,
n = 1,000,000 nodes, degree exponent 2.3, mean degree 32, adjacency operator,
K = 32 tracked pairs; each update adds 0.5% new nodes with 16
preferential-attachment edges each and deletes 0.1% of the edges uniformly
(so S = 5,000 > L+P = 200 and the RSVD new-node basis of Sec. 3.5 is used,
L = P = 100).  One step = one full G-REST update (graph update, basis,
projection, eigensolve, lift, and for the mixed arms the FP64 refinement)
through the library's C ABI.  Three arms run the same stream from the same
initial pairs: FP64, MIXED (the headline: FP32 blocks on the tensor cores,
FP64 Cholesky, eigensolves and refinement) and MIXED_FAST (FP32 projected
problems, double-float refinement); the mixed arms' accuracy against the
FP64 arm is part of the line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grest|reference]
                    [--workload cl1m|cl200k|sbm2k]

`value` times K steps with the update batches already resident in device
memory; `e2e` times K further steps through the same public call with the
batches in pinned host memory (host->device copies inside the timed region)
and a device->host read of the updated embedding (U and theta) after every
step, started without waiting (grest_get_embedding_async) so that it
overlaps the next update; every read completes inside the timed region.  Under torchrun every rank runs an independent replica (the update
does not shard; there is no collective on the data path) and rank 0 prints
the line.  --workload cl200k / sbm2k run the other two single-graph
workloads (FP64, with the oracle timed beside them).
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G-REST updates/s at n=1M,k=32: mixed vs FP64 GPU path; p50/p99 update latency"
WL = dict(n=1_000_000, gamma=2.3, mean_degree=32, k=32, grow_frac=0.005, edges_per_new_node=16,
          delete_frac=0.001, seed=20260306, L=100, P=100)
# the three single-graph workloads: the 1M-node adjacency stream (the
# headline), the 200k-node normalized-Laplacian stream and the SBM stream
WORKLOADS = {
    "cl1m": dict(kind="power_law", n=1_000_000, gamma=2.3, mean_degree=32, k=32, op=0, lcc=False, grow_frac=0.005,
                 edges_per_new_node=16, delete_frac=0.001, seed=20260306, L=100, P=100,
                 precisions=("fp64", "mixed", "mixed_fast"), metric=METRIC),
    "cl200k": dict(kind="power_law", n=200_000, gamma=2.5, mean_degree=16, k=16, op=2, lcc=True, grow_frac=0.005,
                   edges_per_new_node=8, delete_frac=0.001, seed=20260305, L=100, P=100, precisions=("fp64",),
                   metric="G-REST updates/s, Chung-Lu n=200k normalized Laplacian k=16, FP64 GPU path"),
    "sbm2k": dict(kind="sbm", n=2000, n_comm=4, p_in=0.05, p_out=0.005, k=8, op=0, n_new=50, n_rand=200,
                  seed=20260304, L=100, P=100, precisions=("fp64",),
                  metric="G-REST updates/s, SBM n=2,000 4 communities k=8, FP64 GPU path"),
}
# seconds of timed oracle work per CPU leg (bounded sample of the workload)
CPU_BUDGET_S = 60.0
# pivots of an FP32-accumulated Gram are resolved only to ~5e-4 R_00, so the mixed path drops below 1e-3
MIXED_DROP_TOL = 1e-3
# FP64 peak derived from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values of x (every rank gets it): the
    slowest replica's time sets the whole job's time."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return tt.item()


def replica_rate(t_local, steps, world, device="cuda"):
    """(job time, whole-job updates/s) of `world` replicas that each applied
    `steps` updates, rank r in t_local seconds: every replica's updates count,
    over the slowest replica's time."""
    t = max_over_ranks(t_local, world, device)
    return t, world * steps / t


OP_NAMES = {0: "adjacency", 1: "shifted Laplacian", 2: "normalized Laplacian"}


def workload_desc(w, n=None):
    n = n or w["n"]
    if w["kind"] == "sbm":
        return (f"SBM stream n={n:,} {w['n_comm']} equal communities p_in={w['p_in']} p_out={w['p_out']} "
                f"{OP_NAMES[w['op']]} K={w['k']}, +{w['n_new']} nodes and +{w['n_rand']} random edges per step, "
                f"exact new-node block")
    return (f"Chung-Lu power-law stream n={n:,} gamma={w['gamma']} mean_degree={w['mean_degree']} "
            f"{OP_NAMES[w['op']]}{' (largest component)' if w['lcc'] else ''} K={w['k']}, "
            f"+{w['grow_frac'] * 100:.1f}% nodes x {w['edges_per_new_node']} PA edges and "
            f"-{w['delete_frac'] * 100:.1f}% edges per step, RSVD L=P={w['L']}")


def make_workload(w, steps, seed, n=None):
    """(initial graph, `steps` update batches) of workload w."""
    from paper_2603_19439_gb300 import workloads as wl
    if w["kind"] == "sbm":
        return wl.sbm_stream(seed=seed, n0=n or w["n"], n_comm=w["n_comm"], p_in=w["p_in"], p_out=w["p_out"],
                             steps=steps, n_new=w["n_new"], n_rand=w["n_rand"])
    return wl.power_law_workload(n or w["n"], w["gamma"], w["mean_degree"], steps, w["grow_frac"],
                                 w["edges_per_new_node"], w["delete_frac"], seed, lcc=w["lcc"])


def batches_needed(steps, warmup):
    """Batches of one bench run: W warm-up and K timed steps; the end-to-end
    leg replays the same W + K on a fresh tracker of the headline arm."""
    return warmup + steps


def stream_node_capacity(n0, batches):
    """Node ids after every batch of the stream, plus slack.  Contexts are
    created with this capacity so that no capacity growth (which the library
    does on demand, with device-wide synchronizing frees) lands inside a timed
    region."""
    return int(n0) + sum(int(b.n_new) for b in batches) + 1024


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling (every 200 ms) of SM clocks and throttle reasons."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                if self.bus_id and self.bus_id not in p[1].lower() and p[1].lower() not in self.bus_id:
                    continue
                rows.append(p)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

def oracle_initial_state(w, g):
    """Oracle state at step 0 for a timed CPU sample.  Small graphs take the
    oracle's own direct eigendecomposition.  For the large ones a direct
    solve (ARPACK at n = 1M) alone takes minutes, so the initial basis is a
    Rayleigh-Ritz approximation after four block power iterations (seeded);
    the update step does the same work whatever the accuracy of its input
    basis (the block sizes m = K + r_W + r_B do not depend on it)."""
    import oracle as O
    from paper_2603_19439_gb300 import workloads as wl
    rp, col, val = wl.csr_fast(g)
    K, op = w["k"], w["op"]
    if g.n <= 20_000:
        return O.init_state(g.n, rp, col, val, K, op), "direct eigendecomposition"
    A = O.csr_from_arrays(g.n, rp, col, val)
    live = np.ones(g.n, bool)
    M, _ = O.operator_matrix(A, live, op)
    X = np.random.default_rng(w["seed"]).standard_normal((g.n, K + 8))
    for _ in range(4):
        X, _ = np.linalg.qr(M @ X)
    ev, F = np.linalg.eigh(X.T @ (M @ X))
    order = O.select_order(ev, op)[:K]
    st = O.State(A=A, live=live, X=np.ascontiguousarray(X @ F[:, order]), lam=ev[order], step=0)
    return st, "Rayleigh-Ritz basis after 4 block power iterations"


def oracle_sample(w, max_steps, budget_s=CPU_BUDGET_S, stream=None):
    """Time the FP64 CPU oracle on the workload itself (no size scaling):
    consecutive update steps of the same seeded stream the GPU arm runs, at
    most max_steps of them and no more once budget_s seconds of timed work
    are spent (at least one).  stream: (graph, batches) already generated.
    Returns (seconds per timed step, description of the sample)."""
    import oracle as O
    g, batches = stream if stream is not None else make_workload(w, max(1, max_steps), w["seed"])
    batches = batches[:max(1, max_steps)]
    st, how = oracle_initial_state(w, g)
    cfg = O.Config(k=w["k"], op=w["op"], L=w["L"], P=w["P"], seed=w["seed"])
    times = []
    for b in batches:
        t0 = time.perf_counter()
        st, _ = O.grest_step(st, b, cfg)
        times.append(time.perf_counter() - t0)
        if sum(times) >= budget_s:
            break
    desc = (f"{len(times)} consecutive FP64 oracle update steps of the n={g.n:,} workload itself (no scaling; "
            f"initial basis: {how}); NumPy/SciPy BLAS on all host cores, scipy.sparse products single-threaded; "
            f"bounded at {budget_s:.0f} s of timed work")
    return times, desc


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    times, sample = oracle_sample(w, args.steps)
    t = sum(times)
    value = len(times) / t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": w["metric"], "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w), "precision": "fp64",
                       "steps_requested": args.steps, "warmup_requested": args.warmup,
                       "note": "the oracle is CPU code: it has no warm-up effect, and its steps are a bounded "
                               "sample of the requested ones"},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

# Sources of each kernel kind (GREST_KIND_*): a traffic figure taken with ncu
# counts only while these files are unchanged.
KIND_SOURCES = {
    "spmm_f32": ["paper_2603_19439_gb300/csrc/spmm.cu"],
    "spmm_f64": ["paper_2603_19439_gb300/csrc/spmm.cu"],
    "gram_tc": ["paper_2603_19439_gb300/csrc/tc_gram.cu", "paper_2603_19439_gb300/csrc/tc_util.cuh"],
    "gram_narrow": ["paper_2603_19439_gb300/csrc/narrow_gram.cu"],
    "gram_cuda": ["paper_2603_19439_gb300/csrc/dense.cu"],
    "gemm_tc": ["paper_2603_19439_gb300/csrc/tc_gemm.cu", "paper_2603_19439_gb300/csrc/tc_util.cuh"],
    "gemm_cuda": ["paper_2603_19439_gb300/csrc/dense.cu"],
}
KIND_CLASS = {"spmm_f32": 0, "spmm_f64": 0, "gram_tc": 1, "gram_narrow": 1, "gram_cuda": 1, "gemm_tc": 2,
              "gemm_cuda": 2, "small": 3, "graph": 4}
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "traffic_grest_step_mixed_chung_lu_1M.md")


def read_traffic(path, n_mean):
    """DRAM bytes per launch per kernel kind from an ncu capture summary (its
    table rows: | kind | launches per step | DRAM bytes per launch | mean node
    ids | sources hash |), scaled from the captured steps' mean node count to
    n_mean; a kind whose sources changed since the capture gets none."""
    out = {}
    try:
        text = open(path).read()
    except OSError:
        return out
    for m in re.finditer(r"^\| `?([a-z_0-9]+)`? \| ([0-9.]+) \| ([0-9.]+) \| ([0-9.]+) \| `?([0-9a-f]{16})`? \|$",
                         text, re.M):
        kind, _, per_launch, n_cap, h = m.groups()
        if kind in KIND_SOURCES and source_hash(KIND_SOURCES[kind]) == h and n_mean:
            out[kind] = float(per_launch) * n_mean / float(n_cap)
    return out


def roofline(prof_ms, prof_work, prof_bytes, prof_launch, kinds, n_mean, precision="fp64"):
    """Roofline of the dominant kernel class of the step (by device time),
    with every class and every kernel kind (GREST_KIND_*) listed beside it.

    SpMM, Gram and GEMM are HBM-bound in the mixed path (tensor cores keep the
    products at or below the ridge): achieved = compulsory bytes / time
    against the measured copy bandwidth.  FP64 work (the FP64 path, and in the
    mixed path the refinement's FP64 SpMM, Gram and lift) is FP64-pipe bound:
    flops against the derived FP64 peak; the small dense class is latency /
    ALU bound.  `traffic` (DRAM bytes per launch) comes from the ncu capture
    summary in profiles/ for the kinds whose sources are unchanged; a class
    gets it when every launch of the class is of such a kind."""
    from paper_2603_19439_gb300 import grest as G
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s (of fallback)"
    fp64 = (FP64_PEAK_TFLOPS, "FP64 DFMA: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived)")
    fp32 = (FP32_PEAK_TFLOPS, "FP32 FFMA: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (derived)")

    def fig(bound, ms, work, byts, launches, alu=fp64):
        if ms <= 0:
            return None
        if bound == "hbm":
            r = {"bound": "hbm", "unit": "GB/s", "achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm, "peak_source": hbm_src}
        else:
            r = {"bound": "alu", "unit": "TFLOP/s", "achieved": work / (ms * 1e-3) / 1e12, "peak": alu[0],
                 "peak_source": alu[1]}
        r["frac"] = r["achieved"] / r["peak"]
        r["ms_per_step"] = float(ms)
        r["launches_per_step"] = float(launches)
        return r

    classes = {}
    for c in range(5):
        name = G.PROF_CLASSES[c]
        hbm_bound = name in ("spmm", "graph") or (precision != "fp64" and name in ("gram", "gemm"))
        alu = fp32 if (precision == "mixed_fast" and name == "small") else fp64
        r = fig("hbm" if hbm_bound else "alu", prof_ms[c], prof_work[c], prof_bytes[c], prof_launch[c], alu)
        if r:
            classes[name] = r
    kms, kwork, kbytes, kn = kinds
    fp64_kinds = {"spmm_f64", "gram_cuda", "gemm_cuda"}
    kernels = {}
    for i, name in enumerate(G.PROF_KINDS):
        if name in ("small", "graph", "double_float"):
            continue
        r = fig("alu" if name in fp64_kinds else "hbm", kms[i], kwork[i], kbytes[i], kn[i])
        if r:
            r["kernels"] = G.PROF_KIND_KERNELS[i]
            kernels[name] = r
    traffic = read_traffic(TRAFFIC_PROFILE, n_mean)
    for name, r in kernels.items():
        r["traffic"] = traffic.get(name)
    for cname, r in classes.items():
        c = G.PROF_CLASSES.index(cname)
        ks = [k for k, cc in KIND_CLASS.items() if cc == c and k in kernels]
        covered = sum(kernels[k]["launches_per_step"] for k in ks)
        r["traffic"] = None
        if ks and abs(covered - r["launches_per_step"]) < 0.5 and all(kernels[k]["traffic"] is not None for k in ks):
            r["traffic"] = sum(kernels[k]["traffic"] * kernels[k]["launches_per_step"] for k in ks) / covered
    cls = int(np.argmax(prof_ms))
    name = G.PROF_CLASSES[cls]
    out = dict(classes.get(name, {}))
    out.update({"kernel_class": name, "traffic": classes.get(name, {}).get("traffic"), "classes": classes,
                "kernels": kernels,
                "traffic_source": "profiles/traffic_grest_step_mixed_chung_lu_1M.md (ncu DRAM bytes per launch, "
                                  "scaled to this run's mean node count; null where the kernel changed since)"})
    return out


def source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(ROOT, f)
        if not os.path.exists(p):
            return None
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def initial_pairs(tr, n, k, torch):
    """Leading K pairs of A^(0) (the initial pairs of Alg. 2, from a direct eigensolver):
    ARPACK Lanczos whose products A x run in the library's SpMM."""
    import scipy.sparse.linalg as ssl
    x_d = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    y_d = torch.empty_like(x_d)

    def mv(x):
        x_d.copy_(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).reshape(n, 1)))
        tr.apply_operator(x_d, y_d)
        return y_d.cpu().numpy().reshape(-1)

    op = ssl.LinearOperator((n, n), matvec=mv, dtype=np.float64)
    ev, V = ssl.eigsh(op, k=k + 8, which="LM", tol=1e-10, v0=np.ones(n))
    order = sorted(range(ev.size), key=lambda i: (-abs(ev[i]), -ev[i], i))[:k]
    return np.ascontiguousarray(V[:, order]), ev[order]


def pair_diagnostics(tr, U, theta, torch):
    """Residuals of the tracked pairs on the current graph: per pair
    ||M u - theta u|| / |theta_1| with M u from the library's FP64 SpMM
    (grest_apply_operator); the Galerkin residual max |U^T (M U - U Theta)|
    / |theta_1| and the orthonormality max |U^T U - I|.  Diagnostics of the
    bench line only (outside every timed region)."""
    X = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    Y = torch.empty_like(X)
    tr.apply_operator(X, Y)
    th = torch.from_numpy(np.ascontiguousarray(theta)).cuda()
    R = Y - X * th
    scale = float(abs(theta[0]))
    res = (torch.linalg.vector_norm(R, dim=0) / scale).cpu().numpy()
    gal = float((X.T @ R).abs().max()) / scale
    orth = float((X.T @ X - torch.eye(X.shape[1], dtype=X.dtype, device=X.device)).abs().max())
    del X, Y, R
    return {"residual": res, "galerkin": gal, "orth_err": orth}


def subspace_sin(Ua, Ub, torch):
    """Sine of the largest principal angle between span(Ua) and span(Ub)
    (both orthonormal): the 2-norm of Ub - Ua (Ua^T Ub)."""
    if Ua.shape[1] == 0:
        return 0.0
    A = torch.from_numpy(np.ascontiguousarray(Ua)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(Ub)).cuda()
    P = B - A @ (A.T @ B)
    ev = torch.linalg.eigvalsh(P.T @ P)
    return float(max(float(ev[-1]), 0.0) ** 0.5)


def cluster_cut(theta, op, gap=1e-6):
    """Largest j <= K such that tracked values j-1 and j are separated by more
    than gap * |theta_1| (in the tracking order: |theta| for the adjacency)."""
    key = np.abs(theta) if op == 0 else np.asarray(theta)
    scale = max(abs(theta[0]), 1e-300)
    for j in range(len(theta), 0, -1):
        if j == len(theta) or abs(key[j - 1] - key[j]) > gap * scale:
            return j
    return 0


PRECISIONS = {"fp64": ("FP64", 1e-7), "mixed": ("MIXED", 1e-3), "mixed_fast": ("MIXED_FAST", 1e-3)}
PRECISION_DESC = {
    "fp64": "FP64 blocks, products, projected problems",
    "mixed": "FP32 blocks, FP32 SpMM, 3xTF32 tensor-core Grams / block updates with FP64 partial sums; FP64 "
             "pivoted Cholesky, FP64 m x m and RSVD eigensolves, FP64 Rayleigh-Ritz refinement in span(U) "
             "(FP64 SpMM of U, FP64 Grams and lift)",
    "mixed_fast": "as mixed, but FP32 pivoted Cholesky and eigensolves, and the refinement's N x K products in "
                  "double-float (FP32 hi + lo) arithmetic",
}


def run_grest(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_19439_gb300 import grest as G
    from paper_2603_19439_gb300 import workloads as wl

    w = WORKLOADS[args.workload]
    n, K, W, steps = args.nodes or w["n"], w["k"], args.warmup, args.steps
    precs = [p for p in w["precisions"] if not (args.fp64_only and p != "fp64") and
             not (args.mixed_only and p == "fp64") and not (args.no_fast and p == "mixed_fast")]
    if not precs:
        raise SystemExit("no precision arm selected")
    headline = "mixed" if "mixed" in precs else precs[0]
    t0 = time.time()
    g, batches = make_workload(w, batches_needed(steps, W), w["seed"] + 1000 * rank, n=n)
    rp, col, val = wl.csr_fast(g)
    t_gen = time.time() - t0
    stream = torch.cuda.current_stream()
    t0 = time.time()
    common = dict(stream=stream.cuda_stream, op=w["op"], L=w["L"], P=w["P"], seed=w["seed"], flags=G.FLAG_PROFILE,
                  node_capacity=stream_node_capacity(g.n, batches))
    if args.init == "device":
        # the library's own FP64 block Krylov solver (grest_init without U0 / theta0)
        tr64 = G.Tracker(g.n, rp, col, val, None, None, K, precision=G.FP64, **common)
        torch.cuda.synchronize()
        t_pairs = time.time() - t0
        U0, th0, _ = tr64.embedding()
    else:
        tr64 = G.Tracker(g.n, rp, col, val, np.zeros((g.n, K)), np.zeros(K), K, precision=G.FP64, **common)
        U0, th0 = initial_pairs(tr64, g.n, K, torch)
        tr64.set_embedding(U0, th0)
        t_pairs = time.time() - t0

    def dev_batch(b):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
        return wl.Batch(b.n_new, t(b.ins_u), t(b.ins_v), t(b.del_u), t(b.del_v), t(b.del_nodes))

    def pinned_batch(b):
        def p(a):
            x = torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()
            return x.numpy()
        return wl.Batch(b.n_new, p(b.ins_u), p(b.ins_v), p(b.del_u), p(b.del_v), p(b.del_nodes))

    dev = [dev_batch(b) for b in batches[:W + steps]]
    host = [pinned_batch(b) for b in batches[W:W + steps]]
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    bus = None
    if hasattr(props, "pci_bus_id"):
        bus = "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id, props.pci_device_id)

    def timed(tr):
        """Warm-up, then K timed steps with device-resident batches."""
        for b in dev[:W]:
            tr.update(b, on_device=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        prof = {"ms": np.zeros(5), "work": np.zeros(5), "bytes": np.zeros(5), "n": np.zeros(5), "launches": 0,
                "kms": np.zeros(10), "kwork": np.zeros(10), "kbytes": np.zeros(10), "kn": np.zeros(10), "nodes": 0.0}
        clocks = ClockSampler(bus)
        clocks.start()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = None
        for i, b in enumerate(dev[W:]):
            ev[i][0].record(stream)
            s = tr.update(b, on_device=True)
            ev[i][1].record(stream)
            prof["ms"] += s["prof_ms"]
            prof["work"] += s["prof_work"]
            prof["bytes"] += s["prof_bytes"]
            prof["n"] += s["prof_launches"]
            prof["launches"] += s["kernel_launches"]
            prof["kms"] += s["prof_kind_ms"]
            prof["kwork"] += s["prof_kind_work"]
            prof["kbytes"] += s["prof_kind_bytes"]
            prof["kn"] += s["prof_kind_launches"]
            prof["nodes"] += s["n_nodes"]
            last = s
        e1.record(stream)
        barrier()
        clk = clocks.stop()
        t = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world)
        lat = sorted(a.elapsed_time(b) for a, b in ev)
        return dict(t=t, lat=lat, prof=prof, last=last, clk=clk)

    t_init = time.time() - t0
    results, tr_head = {}, None
    for p in precs:
        name, tol = PRECISIONS[p]
        tr = tr64 if p == "fp64" else G.Tracker(g.n, rp, col, val, U0, th0, K, precision=getattr(G, name),
                                                drop_tol=tol, **common)
        r = timed(tr)
        r["U"], r["theta"], _ = tr.embedding()
        r["diag"] = pair_diagnostics(tr, r["U"], r["theta"], torch)
        results[p] = r
        if tr is not tr64:
            tr.close()
    tr64.close()
    # ---- end to end through the public call from pinned host memory (headline arm)
    # A fresh tracker of the headline arm replays the same steps as the timed
    # region (W device-batch warm-up steps, then the K timed batches from
    # pinned host memory), so e2e and value cover the same graph sizes.  Every
    # step's pairs are read into pinned host memory with
    # grest_get_embedding_async, so the copy of step t overlaps update t + 1
    # (two host buffers, used in turn; all reads complete inside the region).
    name, tol = PRECISIONS[headline]
    tr_head = G.Tracker(g.n, rp, col, val, U0, th0, K, precision=getattr(G, name), drop_tol=tol, **common)
    for b in dev[:W]:
        tr_head.update(b, on_device=True)
    cap = stream_node_capacity(g.n, batches)
    U_h = [torch.empty((cap, K), dtype=torch.float64).pin_memory() for _ in range(2)]
    theta_h = [torch.empty(K, dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = d2h = 0
    barrier()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for i, b in enumerate(host):
        tr_head.update(b, on_device=False)
        tr_head.wait_embedding()  # the read of step i - 2 (done by now) frees its buffer
        rows = tr_head.embedding_async(U_h[i % 2], theta_h[i % 2])
        h2d += 4 * (2 * b.n_ins + 2 * b.n_del + b.del_nodes.size)
        d2h += 8 * (rows * K + K)
    tr_head.wait_embedding()
    e3.record(stream)
    barrier()
    t_e2e = max_over_ranks(e2.elapsed_time(e3) * 1e-3, world)
    tr_head.close()
    if rank != 0:
        return 0

    r64 = results.get("fp64")

    def accuracy(r):
        d = r["diag"]
        out = {"max_residual": float(d["residual"].max()), "galerkin": d["galerkin"], "orth_err": d["orth_err"],
               "norm": "residuals / |theta_1| with M u from the library's FP64 SpMM, after the last timed step"}
        if r64 is not None and r is not r64:
            th, th64 = r["theta"], r64["theta"]
            j = cluster_cut(th64, w["op"])
            out.update({
                "theta_rel_vs_fp64": float(np.max(np.abs(th - th64)) / abs(th64[0])),
                "sin_angle_vs_fp64": subspace_sin(r64["U"], r["U"], torch),
                "sin_angle_vs_fp64_cut": subspace_sin(r64["U"][:, :j], r["U"][:, :j], torch), "cut": j,
                "residual_diff_vs_fp64": float(np.max(np.abs(d["residual"] - r64["diag"]["residual"]))),
                "m": r["last"]["m"], "m_fp64": r64["last"]["m"]})
        return out

    def summary(p, r):
        return {"updates_per_s": world * steps / r["t"], "ms_per_step": 1e3 * r["t"] / steps,
                "p50_ms": float(np.percentile(r["lat"], 50)), "p99_ms": float(np.percentile(r["lat"], 99)),
                "precision": PRECISION_DESC[p], "drop_tol": PRECISIONS[p][1],
                "phase_ms_per_step": {G.PROF_CLASSES[i]: float(r["prof"]["ms"][i] / steps) for i in range(5)},
                "kernel_launches_per_step": r["prof"]["launches"] / steps,
                "last_step": {k: r["last"][k] for k in ("m", "rank_q", "rank_y", "mode", "n_nodes", "nnz",
                                                        "pivot_kept_min", "boundary_gap", "ms_refine")},
                "accuracy": accuracy(r),
                "roofline": roofline(r["prof"]["ms"] / steps, r["prof"]["work"] / steps, r["prof"]["bytes"] / steps,
                                     r["prof"]["n"] / steps,
                                     tuple(r["prof"][k] / steps for k in ("kms", "kwork", "kbytes", "kn")),
                                     r["prof"]["nodes"] / steps, p),
                "clocks": r["clk"]}

    main = results[headline]
    arms = {p: summary(p, r) for p, r in results.items()}
    value = world * steps / main["t"]
    res = {
        "metric": w["metric"], "value": value, "unit": "updates/s", "n_gpus": world, "steps": steps, "warmup": W,
        "ms_per_step": 1e3 * main["t"] / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if headline == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": workload_desc(w, n), "precision": headline,
                   "precision_detail": PRECISION_DESC[headline], "k": K, "n0": g.n,
                   "nnz0": int(rp[-1]), "l2": "inputs larger than L2 (graph and N x m blocks are GBs); no flush"
                   if g.n >= 200_000 else "inputs smaller than L2; no flush (the step is launch-bound)",
                   "parallelism": f"replicas{world}", "node_capacity": common["node_capacity"]},
        "latency_ms": {"p50": float(np.percentile(main["lat"], 50)), "p99": float(np.percentile(main["lat"], 99)),
                       "min": main["lat"][0], "max": main["lat"][-1]},
        "accuracy": arms[headline]["accuracy"],
        "arms": arms,
        "e2e": {"value": world * steps / t_e2e, "unit": "updates/s", "h2d_bytes_per_step": h2d // steps,
                "d2h_bytes_per_step": d2h // steps, "precision": headline,
                "returns": "U (N' x K FP64) and theta after every step, read with grest_get_embedding_async into "
                           "pinned host memory (overlapping the next update); all reads complete inside the region"},
        "gpu_launches": int(main["prof"]["launches"]),
        "roofline": arms[headline]["roofline"],
        "clocks": main["clk"],
        "init_s": {"generate": t_gen, "initial_pairs": t_pairs, "initial_pairs_method":
                   "device block Krylov" if args.init == "device" else "ARPACK on the library SpMM",
                   "contexts": t_init},
    }
    if "fp64" in arms and headline != "fp64":
        res["roofline_fp64"] = arms["fp64"]["roofline"]
    if not args.no_cpu_baseline and world == 1:
        times, sample = oracle_sample(w, steps, stream=(g, batches))
        ups = len(times) / sum(times)
        res["cpu_baseline"] = {"value": ups, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": sample}
    print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_kernels(args):
    """--kernels: CUDA-event times of the mixed path's Gram and GEMM entry
    points (grest_gram_f32, grest_gemm_f32; each picks its kernel by shape:
    the narrow CUDA-core Gram for a side of at most 32 columns, else the
    tensor cores) on n x w FP32 blocks of the widths one 1M-node update uses;
    one JSON line (not the bench contract's)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_19439_gb300 import grest as G
    from paper_2603_19439_gb300 import workloads as wl
    torch.cuda.set_device(0)
    g, _ = wl.sbm_graph(200, 2, 0.1, 0.02, 71)
    rp, col, _ = g.csr()
    X0 = np.linalg.qr(np.random.default_rng(0).standard_normal((200, 4)))[0]
    tr = G.Tracker(g.n, rp, col, None, X0, np.ones(4), 4)
    n, reps, out = args.nodes or WL["n"], 10, {"gram": [], "gemm": []}

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for a, b, sym in [(32, 32, False), (32, 232, False), (200, 200, True), (232, 232, True), (164, 164, False)]:
        X = torch.randn((n, a), dtype=torch.float32, device="cuda")
        Y = X if sym else torch.randn((n, b), dtype=torch.float32, device="cuda")
        C = torch.empty((a, b), dtype=torch.float64, device="cuda")
        ms = timed(lambda: tr.gram_f32(X, Y, C))
        by = n * (a + (0 if sym else b)) * 4
        out["gram"].append({"a": a, "b": b, "X_is_Y": sym, "ms": ms, "GB/s": by / ms / 1e6})
        del X, Y
    for a, c, beta in [(32, 232, 1.0), (232, 232, 0.0), (200, 200, 0.0), (232, 132, 0.0), (164, 32, 0.0)]:
        X = torch.randn((n, a), dtype=torch.float32, device="cuda")
        B = torch.randn((a, c), dtype=torch.float64, device="cuda")
        O = torch.randn((n, c), dtype=torch.float32, device="cuda")
        ms = timed(lambda: tr.gemm_f32(X, B, O, 1.0, beta, O if beta else None))
        by = n * (a + c * (2 if beta else 1)) * 4
        out["gemm"].append({"a": a, "c": c, "beta": beta, "ms": ms, "GB/s": by / ms / 1e6})
        del X, B, O
    tr.close()
    print(json.dumps({"kernels": out, "n": n, "reps": reps, "unit": "ms per call (CUDA events, warm)"}), flush=True)
    return 0


def run_batched(args):
    """--batched: many small SBM graphs updated together.  Graph i: n
    log-uniform on [1,000, 50,000], R uniform on {2..16} equal communities,
    mean degree uniform on [8, 24] with p_in = 10 p_out; K = 8, L = P = 20,
    FP64.  One round = one update for every graph: +1% nodes, 1% of the edges
    deleted and as many random edges inserted.  Engine `group` (default):
    grest_group_* -- one grouped launch per stage for all graphs, the update
    captured as a CUDA graph, launch shapes autotuned after the first round.
    Engine `contexts`: one context per graph on its own stream, stepped by
    the library's host threads (grest_batch_*).  Prints one JSON line."""
    import threading
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_19439_gb300 import grest as G
    from paper_2603_19439_gb300 import workloads as wl
    torch.cuda.set_device(0)
    ng, K = args.graphs, 8
    rounds, warm = max(1, args.steps), max(3, args.warmup)
    rng = np.random.default_rng(20260307)
    t0 = time.time()
    graphs = []
    for i in range(ng):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(50000))))
        R = int(rng.integers(2, 17))
        d = rng.uniform(8, 24)
        p_out = d / (n * (1.0 + 9.0 / R))
        graphs.append(wl.sbm_graph(n, R, min(1.0, 10 * p_out), p_out, 20260307 + i)[0])
    batches = [[] for _ in range(ng)]
    for i, g in enumerate(graphs):
        gb = g.copy()
        for _ in range(warm + rounds):
            m = gb.n_edges
            b = wl.random_churn_batch(gb, max(1, gb.n // 100), max(1, m // 100), max(1, m // 100), rng)
            gb.apply(b)
            batches[i].append(b)
    t_gen = time.time() - t0
    t0 = time.time()
    streams = [torch.cuda.Stream() for _ in range(ng)]
    trackers = [None] * ng
    nxt = [0]
    lock = threading.Lock()
    grouped = args.batched_engine == "group"

    def make():
        while True:
            with lock:
                i = nxt[0]
                nxt[0] += 1
            if i >= ng:
                return
            g = graphs[i]
            rp, col, val = g.csr()
            extra = dict(precision=G.MIXED, drop_tol=MIXED_DROP_TOL) if args.batched_precision == "mixed" else {}
            trackers[i] = G.Tracker(g.n, rp, col, val, None, None, K, stream=streams[i].cuda_stream, L=20, P=20,
                                    node_capacity=stream_node_capacity(g.n, batches[i]), **extra)

    pool = [threading.Thread(target=make) for _ in range(args.threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    group = None
    if grouped:
        blobs = [tr.checkpoint() for tr in trackers]
        for tr in trackers:
            tr.close()
        trackers = []
        group = G.Group(blobs, capacity_factor=1.0 + 0.02 * (warm + rounds) + 0.05)
    t_init = time.time() - t0

    def dev(b):
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
        return wl.Batch(b.n_new, c(b.ins_u), c(b.ins_v), c(b.del_u), c(b.del_v), c(b.del_nodes))

    if grouped:
        for r in range(warm):
            codes, _ = group.update([batches[i][r] for i in range(ng)])
            assert all(c == 0 for c in codes), codes
        info = group.info()
        times, lat = [], []
        for r in range(rounds):
            t = time.perf_counter()
            codes, stats = group.update([batches[i][warm + r] for i in range(ng)])
            times.append(time.perf_counter() - t)
            assert all(c == 0 for c in codes), codes
        info = group.info()
        note = ("grouped: one launch per stage for all graphs (%d launches per update of the group), replayed as "
                "one CUDA graph; autotuned SpMM grid %d x %d rows per warp, GEMM grid %d; the timed region "
                "includes packing and copying the host batches in and reading every graph's state back"
                % (info["launches_per_update"], info["spmm_blocks"], info["spmm_rows_per_warp"],
                   info["gemm_blocks"]))
        step_lat = None
    else:
        batch = G.Batch(trackers, n_threads=args.threads)
        for r in range(warm):
            batch.update([batches[i][r] for i in range(ng)])
        dev_rounds = [[dev(batches[i][warm + r]) for i in range(ng)] for r in range(rounds)]
        torch.cuda.synchronize()
        times, lat = [], []
        for r in range(rounds):
            t = time.perf_counter()
            codes, stats = batch.update(dev_rounds[r], on_device=True)
            times.append(time.perf_counter() - t)
            lat += [s["ms_total"] for s in stats]
        batch.close()
        info = None
        note = "one context per graph on its own stream, stepped by the library's host threads; not grouped"
        step_lat = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}
    upd = ng * rounds / sum(times)
    nodes = sum(g.n for g in graphs)
    line = {"metric": f"G-REST batched updates/s, {ng} SBM graphs (n 1k-50k log-uniform), K=8, one update each",
            "value": upd, "unit": "updates/s", "n_gpus": 1, "rounds": rounds, "warmup_rounds": warm,
            "ms_per_round": 1e3 * sum(times) / rounds,
            "round_ms": {"p50": float(np.percentile(np.array(times) * 1e3, 50)),
                         "max": float(np.max(times) * 1e3)},
            "higher_is_better": True, "engine": args.batched_engine,
            "dtype": "f64" if (grouped or args.batched_precision == "fp64") else "f32+f64",
            "data": "synthetic", "threads": None if grouped else args.threads,
            "step_latency_ms": step_lat, "group_info": info,
            "config": {"workload": "batched SBM", "graphs": ng, "total_nodes": nodes, "K": K, "L": 20, "P": 20,
                       "update": "+1% nodes, 1% edges deleted and 1% inserted"},
            "setup_s": {"generate": t_gen, "contexts_initial_pairs_and_group": t_init},
            "note": note}
    if group is not None:
        group.close()
    for tr in trackers:
        tr.close()
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """--serve: the serving loop (grest_server_*) under a Poisson stream of
    update requests for many resident Chung-Lu graphs.  Graph i: n
    log-uniform on [--serve-nmin, --serve-nmax] (10,000 .. 2,000,000), mean
    degree 16, gamma 2.3, K uniform on {16..32}.  A request carries E edges,
    E log-uniform on [100, --serve-emax] (100,000; capped at 10% of the
    graph's edges): a quarter attaches new nodes (8 edges each), half are
    uniform inserts, a quarter uniform deletes.  Each precision arm (mixed,
    then FP64) serves the same graphs from the same initial pairs and the
    same requests: one calibration round (one request per graph at once,
    admissions included) sets the sustained rate, and the measured stream
    arrives as a Poisson process at 80% of it.  Latency = arrival ->
    completion.  With --hbm-budget-gb below the resident total, graphs are
    admitted as memory frees up (--evict: idle graphs are checkpointed to
    host memory).  One JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_19439_gb300 import grest as G
    from paper_2603_19439_gb300 import workloads as wl
    torch.cuda.set_device(0)
    ng, nreq = args.graphs, args.requests
    rng = np.random.default_rng(20260308)
    t0 = time.time()
    graphs, ks = [], []
    for i in range(ng):
        n = int(np.exp(rng.uniform(np.log(args.serve_nmin), np.log(args.serve_nmax))))
        graphs.append(wl.chung_lu_graph(n, 2.3, 16, 20260308 + i))
        ks.append(int(rng.integers(16, 33)))
    # requests: a calibration round (one per graph) and then nreq Poisson arrivals
    order = [i for i in range(ng)] + [int(x) for x in rng.integers(0, ng, size=nreq)]
    copies = [g.copy() for g in graphs]
    reqs = []
    for gi in order:
        gb = copies[gi]
        E = int(np.exp(rng.uniform(np.log(100), np.log(args.serve_emax))))
        E = max(8, min(E, gb.n_edges // 10))
        b = wl.random_churn_batch(gb, max(1, E // 32), E // 2, E // 4, rng, new_edges_per_node=8)
        gb.apply(b)
        reqs.append((gi, b))
    del copies
    csrs = [wl.csr_fast(g) for g in graphs]
    t_gen = time.time() - t0
    # initial pairs once per graph (the library's FP64 device solver), shared by both arms
    t0 = time.time()
    pairs = []
    for g, (rp, col, val), k in zip(graphs, csrs, ks):
        tr = G.Tracker(g.n, rp, col, val, None, None, k)
        U0, th0, _ = tr.embedding()
        tr.close()
        pairs.append((U0, th0))
    t_pairs = time.time() - t0
    gaps = rng.exponential(1.0, size=nreq)
    budget = int(args.hbm_budget_gb * 1e9) if args.hbm_budget_gb > 0 else 1 << 50
    arms = {}
    for prec in args.serve_precisions.split(","):
        sv = G.Server(n_workers=args.threads, hbm_budget=budget)
        if args.evict:
            sv.set_eviction(True)
        extra = dict(precision=G.MIXED, drop_tol=MIXED_DROP_TOL) if prec == "mixed" else {}
        gids = [sv.add_graph(g.n, rp, col, val, k, U0=U0, theta0=th0,
                             node_capacity=stream_node_capacity(g.n, [b for gi, b in reqs if gi == i]), **extra)
                for i, (g, (rp, col, val), k, (U0, th0)) in enumerate(zip(graphs, csrs, ks, pairs))]
        # calibration: one request per graph at once (admissions happen here)
        tc = time.perf_counter()
        cal = [sv.submit(gids[gi], b) for gi, b in reqs[:ng]]
        cal_codes = [sv.wait(t)[0] for t in cal]
        t_cal = time.perf_counter() - tc
        cap = ng / t_cal
        rate = 0.8 * cap
        stream = reqs[ng:]
        arrivals, tickets = [], []
        start = time.perf_counter()
        for (gi, b), gap in zip(stream, gaps / rate):
            target = (arrivals[-1] if arrivals else start) + gap
            now = time.perf_counter()
            if target > now:
                time.sleep(target - now)
            arrivals.append(time.perf_counter())
            tickets.append(sv.submit(gids[gi], b))
        lat, codes, runs = [], [], []
        for t in tickets:
            code, _, wait_ms, run_ms = sv.wait(t)
            codes.append(code)
            lat.append(wait_ms + run_ms)
            runs.append(run_ms)
        wall = time.perf_counter() - start
        used, nres = sv.resident()
        adm, evc, rst = sv.counters()
        arms[prec] = {"updates_per_s": len(stream) / wall, "arrival_rate_per_s": rate, "sustained_rate_per_s": cap,
                      "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                     "max": float(np.max(lat))},
                      "run_ms": {"p50": float(np.percentile(runs, 50)), "p99": float(np.percentile(runs, 99))},
                      "failed": int(sum(c != 0 for c in codes) + sum(c != 0 for c in cal_codes)),
                      "resident_graphs_at_end": nres, "resident_bytes_at_end": used,
                      "admissions": adm, "evictions": evc, "restores": rst,
                      "calibration_round_s": t_cal}
        sv.close()
    head = "mixed" if "mixed" in arms else next(iter(arms))
    line = {"metric": f"G-REST serving: {ng} resident Chung-Lu graphs, Poisson update requests",
            "value": arms[head]["updates_per_s"], "unit": "updates/s", "n_gpus": 1, "requests": nreq,
            "higher_is_better": True, "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
            "workers": args.threads, "precision": head,
            "latency_ms": arms[head]["latency_ms"], "arms": arms,
            "hbm_budget_bytes": budget if args.hbm_budget_gb > 0 else None, "eviction": bool(args.evict),
            "config": {"workload": "serving Chung-Lu", "graphs": ng, "nodes_total": int(sum(g.n for g in graphs)),
                       "nodes_min": int(min(g.n for g in graphs)), "nodes_max": int(max(g.n for g in graphs)),
                       "K": "16..32", "edges_per_request": f"100..{args.serve_emax:,} log-uniform (<= 10% of the graph)"},
            "setup_s": {"generate": t_gen, "initial_pairs": t_pairs},
            "note": "latency = arrival -> completion; the calibration round (admissions) is not in the measured "
                    "stream; both arms serve the same graphs, initial pairs and requests"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["grest", "reference"], default="grest")
    ap.add_argument("--init", choices=["device", "arpack"], default="device",
                    help="initial pairs: the library's device solver, or host ARPACK over the library SpMM")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", action="store_true", help="many small SBM graphs through grest_batch_apply_updates")
    ap.add_argument("--graphs", type=int, default=512, help="--batched: number of graphs")
    ap.add_argument("--batched-precision", choices=["fp64", "mixed"], default="fp64", help="--batched / --serve: step precision")
    ap.add_argument("--threads", type=int, default=16, help="--batched: host threads")
    ap.add_argument("--batched-engine", choices=["group", "contexts"], default="group",
                    help="--batched: grouped launches under CUDA-graph capture, or one context per graph")
    ap.add_argument("--serve", action="store_true", help="the serving loop under Poisson update requests")
    ap.add_argument("--requests", type=int, default=256, help="--serve: measured requests")
    ap.add_argument("--serve-nmin", type=int, default=10_000, help="--serve: smallest graph (log-uniform sizes)")
    ap.add_argument("--serve-nmax", type=int, default=2_000_000, help="--serve: largest graph")
    ap.add_argument("--serve-emax", type=int, default=100_000, help="--serve: largest request (edges)")
    ap.add_argument("--serve-precisions", default="mixed,fp64", help="--serve: arms, in order")
    ap.add_argument("--hbm-budget-gb", type=float, default=0.0,
                    help="--serve: device-memory budget of the resident graphs (0 = unlimited)")
    ap.add_argument("--evict", action="store_true",
                    help="--serve: checkpoint idle graphs to host memory when a waiting graph does not fit")
    ap.add_argument("--kernels", action="store_true",
                    help="time the mixed path's Gram / GEMM entry points at the step's widths instead")
    ap.add_argument("--fp64-only", action="store_true", help="skip the mixed-precision arms")
    ap.add_argument("--mixed-only", action="store_true", help="skip the FP64 arm")
    ap.add_argument("--no-fast", action="store_true", help="skip the MIXED_FAST arm")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cl1m",
                    help="cl1m: the 1M-node adjacency stream (default); cl200k: 200k-node normalized Laplacian; "
                         "sbm2k: the SBM stream")
    ap.add_argument("--nodes", type=int, default=None,
                    help="graph size of the same workload family (smaller sizes are for profiler captures; "
                         "the reported metric is defined at the workload's own size)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.kernels:
        return run_kernels(args)
    if args.batched:
        return run_batched(args)
    if args.serve:
        return run_serve(args)
    return run_grest(args)


if __name__ == "__main__":
    sys.exit(main())
