#!/usr/bin/env python
"""Benchmark of the GB300 ParIS+ hot path on random-walk data (ParIS+ Sec. 4 workload shape).

Workload (one step): build the iSAX index of 20,000,000 z-normalised random-walk series of
length 256 (fp32, w = 16, 8-bit symbols) that are already resident in HBM, then answer exact
1-NN for 3,000 queries -- 1,000 noisy copies of dataset rows for each noise level
sigma in {0.01, 0.1, 1.0}. value = queries answered per second of step time (build included).

Prints one JSON line. ``--impl reference`` times the CPU oracle (FP64 brute force with exact
re-ranking) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact 1-NN queries/s at 20M×256 fp32; build GB/s; LB-scan % of HBM peak"
SIGMAS = (0.01, 0.1, 1.0)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=20_000_000)
    p.add_argument("--len", type=int, default=256)
    p.add_argument("--per-sigma", type=int, default=1000)
    p.add_argument("--k", type=int, default=1)
    p.add_argument("--mode", default="batched", choices=["plain", "batched"])
    p.add_argument("--precision", default="mixed", choices=["fp32", "mixed"])
    p.add_argument("--seed", default="descent", choices=["descent", "learned"])
    p.add_argument("--no-learned-comparison", action="store_true",
                   help="skip training the seed model and the learned-seed comparison runs")
    p.add_argument("--train-queries", type=int, default=20000, help="(query, true-NN bucket) pairs for the seed model")
    p.add_argument("--train-epochs", type=int, default=10)
    p.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain fp32 method shown beside")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--query-tile", type=int, default=0,
                   help="queries per batched summary pass (0: the library tunes it)")
    p.add_argument("--graph-steps", type=int, default=3,
                   help="timed replays of the captured batch (index built once) shown beside")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="target CPU time of the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--clocks-csv", default="", help="keep the raw nvidia-smi clock samples of the timed region here")
    p.add_argument("--leaf-capacity", type=int, default=0, help="rows per approximate-search leaf (0: 2048)")
    p.add_argument("--no-adaptive", action="store_true",
                   help="skip the adaptive-split leaves comparison (seed from ADS+ adaptive leaves vs the fixed trie)")
    p.add_argument("--batch-n", type=int, default=50_000_000,
                   help="rows of the 4096-query batch workload reported beside (0: skip it)")
    p.add_argument("--multi-scale", type=float, default=1.0,
                   help="size factor of the three-collection workload reported beside (0: skip it)")
    p.add_argument("--learned-study", action="store_true",
                   help="instead of the headline: train the learned seed on 2M labelled pairs over 50M x 256 and "
                        "compare it with the descent seed on 10K held-out queries (one JSON line)")
    p.add_argument("--study-n", type=int, default=50_000_000)
    p.add_argument("--study-pairs", type=int, default=2_000_000)
    p.add_argument("--study-heldout", type=int, default=10_000)
    p.add_argument("--study-epochs", type=int, default=4)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        if path:
            self.path = path
            os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        else:
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_bench_{gpu_index}_", suffix=".csv")
            os.close(fd)
        self.temporary = not path
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            if self.temporary:
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if self.temporary:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n, length, per_sigma, rank, pinned=True):
    import numpy as np
    import torch

    import synth
    host = torch.empty((n, length), dtype=torch.float32, pin_memory=pinned)
    synth.random_walk(n, length, seed=1 + 1000 * rank, out=host.numpy())
    q, sig, src = synth.sigma_queries(host.numpy(), n, length, per_sigma, SIGMAS)
    qhost = torch.from_numpy(np.ascontiguousarray(q))
    if pinned:
        qhost = qhost.pin_memory()
    return host, qhost, sig, src


def bf16_peak_sustained():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path)).get("bf16_tflops_sustained", 1700.0))
    return 1700.0


def cpu_baseline(host_np, queries_np, target_s):
    """The oracle as it stands (FP64 GEMM screening + exact re-rank) on a bounded sample."""
    import numpy as np

    from oracle import knn as oknn
    n = host_np.shape[0]
    per = len(queries_np) // len(SIGMAS)
    sample_q = queries_np[[0, per, 2 * per]]          # one query per sigma level
    probe = min(n, 1 << 20)
    t0 = time.perf_counter()
    oknn.knn_chunked(lambda a, b: host_np[a:b], probe, sample_q, 1)
    t_probe = time.perf_counter() - t0
    rows = int(min(n, max(probe, probe * target_s / max(t_probe, 1e-3))))
    t0 = time.perf_counter()
    oknn.knn_chunked(lambda a, b: host_np[a:b], rows, sample_q, 1)
    t = time.perf_counter() - t0
    per_query_full = t / len(sample_q) * (n / rows)
    return {"value": 1.0 / per_query_full, "unit": "queries/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(sample_q)} queries (one per sigma) over the first {rows} of {n} rows, "
                      f"time scaled by {n / rows:.3g} to the full collection; {t:.1f} s of CPU work"}


def traffic_for(kernel: str, query_tile: int = 0, workload: dict | None = None):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current source (the
    SHA-256 prefix of the kernel's source files, concatenated in the listed order), for the same
    workload sizes and, for the batched scan, with the same query tile."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        table = json.load(open(path))
        d = table.get(f"{kernel}@qt{query_tile}") if query_tile else table.get(kernel)
    except Exception:
        return None
    if not d:
        return None
    if any((workload or {}).get(key) != val for key, val in d.get("workload", {}).items()):
        return None
    import hashlib
    h = hashlib.sha256()
    for name in d.get("sources", [d.get("source")]):
        src = os.path.join(ROOT, "paper_2009_00166_gb300", "csrc", name or "")
        if not name or not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    if h.hexdigest()[:16] != d["source_sha"]:
        return None
    return float(d["bytes_per_launch"]) * (d.get("scale", 1.0))


def timed(fn, stream, reps):
    """Device time of `reps` calls of fn (after one untimed call), ms per call."""
    import torch
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


def run_batch_workload(args, P, host20, model, dev, stream):
    """4096-query batches over 50M x 256 random walks (rows [0, 20M) are the headline collection's;
    sigma ~ U[0.01, 2], seed 5), k in {1, 10}: the batched mixed-precision form with the descent
    and with the learned seed (index built once; batch time), beside the plain GPU method (one query
    per lower-bound pass, fp32 refinement) on the first 512 queries of the batch."""
    import numpy as np
    import torch

    import synth
    n = args.batch_n
    n20 = host20.shape[0]
    t0 = time.perf_counter()
    host = torch.empty((n, 256), dtype=torch.float32, pin_memory=True)
    keep = min(n, n20) if host20.shape[1] == 256 else 0
    if keep:
        host[:keep].copy_(host20[:keep])
    synth.random_walk(n, 256, seed=1, out=host.numpy(), start_row=keep)
    q, sig, _ = synth.mixed_sigma_queries(host.numpy(), n, 256, 4096, 0.01, 2.0, seed=5)
    gen_s = time.perf_counter() - t0
    X = host.to(dev)
    Q = torch.from_numpy(q).to(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    idx = P.paris_build_ex(X, 16, 256, bf16_shadow=True)
    ev[1].record(stream)
    torch.cuda.synchronize()
    out = {"workload": f"{n}x256 random walks, 4096-query batches, sigma ~ U[0.01, 2]", "generate_s": gen_s,
           "build_ms": ev[0].elapsed_time(ev[1]), "by_k": []}
    sub = Q[:512]
    for k in (1, 10):
        head_ms, (hi, _, hst) = timed(lambda: P.paris_exact_knn_ex(idx, Q, k, mode=P.PARIS_MODE_BATCHED,
                                                                    precision=P.PARIS_REFINE_MIXED, want_stats=True),
                                      stream, 2)
        rec = {"k": k, "batched_mixed_queries_per_s": 4096 / (head_ms * 1e-3), "batch_ms": head_ms,
               "dense_queries": hst["dense_queries"], "pages_kept_per_query": hst["pages_kept"] / 4096,
               "candidates_per_query": hst["candidates"] / 4096}
        if model is not None:
            P.paris_attach_seed_model(idx, model, 3)
            lms, (li, _) = timed(lambda: P.paris_exact_knn_ex(idx, Q, k, mode=P.PARIS_MODE_BATCHED,
                                                              precision=P.PARIS_REFINE_MIXED,
                                                              seed=P.PARIS_SEED_LEARNED), stream, 1)
            rec["learned_queries_per_s"] = 4096 / (lms * 1e-3)
            rec["learned_identical_answers"] = bool(torch.equal(li, hi))
        pms, (pi, _) = timed(lambda: P.paris_exact_knn_ex(idx, sub, k, mode=P.PARIS_MODE_PLAIN), stream, 1)
        rec["plain_queries_per_s"] = 512 / (pms * 1e-3)
        rec["plain_identical_answers"] = bool(torch.equal(pi, hi[:512]))
        out["by_k"].append(rec)
    idx.free()
    del X, Q, host
    torch.cuda.empty_cache()
    return out


def run_three_collections(args, P, dev, stream):
    """30M x 128 + 10M x 256 + 2M x 1024 random walks (dataset seeds 11, 12, 13) and 2048 queries
    (683 / 683 / 682, sigma ~ U[0.01, 2], query seeds 111, 112, 113) in one multi-collection call,
    k in {1, 10}, beside the plain GPU method per collection on 96 queries each."""
    import numpy as np
    import torch

    import synth
    f = args.multi_scale
    shapes = [(int(30_000_000 * f), 128, 11, 683), (int(10_000_000 * f), 256, 12, 683),
              (int(2_000_000 * f), 1024, 13, 682)]
    t0 = time.perf_counter()
    hosts, qs = [], []
    for n, length, seed, m in shapes:
        h = torch.empty((n, length), dtype=torch.float32, pin_memory=True)
        synth.random_walk(n, length, seed=seed, out=h.numpy())
        hosts.append(h)
        qs.append(synth.mixed_sigma_queries(h.numpy(), n, length, m, 0.01, 2.0, seed=seed + 100)[0])
    gen_s = time.perf_counter() - t0
    Xs = [h.to(dev) for h in hosts]
    Qs = [torch.from_numpy(q).to(dev) for q in qs]
    idxs = [P.paris_build_ex(X, 16, 256, bf16_shadow=X.shape[1] <= 256) for X in Xs]
    torch.cuda.synchronize()
    out = {"workload": "30Mx128 + 10Mx256 + 2Mx1024 random walks (scaled by %g), 2048 queries in one call" % f,
           "generate_s": gen_s, "by_k": []}
    nq = sum(q.shape[0] for q in qs)
    for k in (1, 10):
        ms, (res, sts) = timed(lambda: P.paris_exact_knn_multi(idxs, Qs, k, precision=P.PARIS_REFINE_MIXED,
                                                               want_stats=True), stream, 2)
        rec = {"k": k, "multi_queries_per_s": nq / (ms * 1e-3), "call_ms": ms,
               "query_tile": sts[0]["query_tile"], "dense_queries": [s_["dense_queries"] for s_ in sts]}
        plain = []
        same = True
        for c, (idx, Q) in enumerate(zip(idxs, Qs)):
            pms, (pi, _) = timed(lambda: P.paris_exact_knn_ex(idx, Q[:96], k, mode=P.PARIS_MODE_PLAIN), stream, 1)
            plain.append(96 / (pms * 1e-3))
            same = same and bool(torch.equal(pi, res[c][0][:96]))
        rec["plain_queries_per_s_per_collection"] = plain
        rec["plain_identical_answers"] = same
        out["by_k"].append(rec)
    for idx in idxs:
        idx.free()
    del Xs, Qs, hosts
    torch.cuda.empty_cache()
    return out


def run_learned_study(args):
    """The learned best-so-far proposal at full size: 50M x 256 random walks (seed 1); 2M training
    pairs (query PAA, 12-bit bucket of its exact nearest neighbour) from queries with sigma ~
    U[0.1, 1.0] (seed 20), labelled by the exact search itself; 10K held-out queries, half at
    sigma 0.1 and half at 1.0 (seeds 30, 31). Per sigma: seed looseness (seed / exact squared
    distance), kept pages and candidates per query and queries/s of the batched mixed form with
    the descent seed and with the learned seed, and of the plain method on 500 queries each."""
    import numpy as np
    import torch

    import paper_2009_00166_gb300 as P
    import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    n = args.study_n
    t0 = time.perf_counter()
    host = torch.empty((n, 256), dtype=torch.float32, pin_memory=True)
    synth.random_walk(n, 256, seed=1, out=host.numpy())
    X = host.to(dev)
    gen_s = time.perf_counter() - t0
    idx = P.paris_build_ex(X, 16, 256, bf16_shadow=True)
    torch.cuda.synchronize()
    # labels from the exact search, in batches
    t0 = time.perf_counter()
    m = args.study_pairs
    tq, _, _ = synth.mixed_sigma_queries(host.numpy(), n, 256, m, 0.1, 1.0, seed=20)
    labels = np.empty(m, np.int32)
    paa = torch.empty((m, 16), dtype=torch.float64, device=dev)
    B = 65536
    for b0 in range(0, m, B):
        Qb = torch.from_numpy(tq[b0:b0 + B]).to(dev)
        rows, _ = P.paris_exact_knn_ex(idx, Qb, 1, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED)
        labels[b0:b0 + B] = P.paris_row_buckets(idx, rows.cpu().numpy()[:, 0])
        paa[b0:b0 + B] = P.paris_encode(Qb, 16, 256, want_paa=True)[2]
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    del tq
    t0 = time.perf_counter()
    md = P.SeedModel(1)
    losses = md.train(paa, torch.from_numpy(labels).to(dev), batch=1024, epochs=args.study_epochs, lr=2e-3,
                      order_seed=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    P.paris_attach_seed_model(idx, md, 3)
    groups = []
    half = args.study_heldout // 2
    for gi, (sigma, seed) in enumerate(((0.1, 30), (1.0, 31))):
        q, _, _ = synth.mixed_sigma_queries(host.numpy(), n, 256, half, sigma, sigma, seed=seed)
        Q = torch.from_numpy(q).to(dev)
        rec = {"sigma": sigma, "queries": half}
        ref = None
        for name, sd in (("descent", P.PARIS_SEED_DESCENT), ("learned", P.PARIS_SEED_LEARNED)):
            _, seeds = P.paris_approx_search(idx, Q, 1, sd)
            ms, (ri, rd, st) = timed(lambda: P.paris_exact_knn_ex(idx, Q, 1, mode=P.PARIS_MODE_BATCHED,
                                                                    precision=P.PARIS_REFINE_MIXED, seed=sd,
                                                                    want_stats=True), stream, 2)
            if ref is None:
                ref = (ri, rd)
            true_sq = rd.double()[:, 0] ** 2
            pms, (pi, _, pst) = timed(lambda: P.paris_exact_knn_ex(idx, Q[:500], 1, mode=P.PARIS_MODE_PLAIN, seed=sd,
                                                                     want_stats=True), stream, 1)
            rec[name] = {"seed_looseness_mean": float((seeds.double() / true_sq.clamp_min(1e-30)).mean()),
                         "batched_mixed_queries_per_s": half / (ms * 1e-3),
                         "pages_kept_per_query": st["pages_kept"] / half,
                         "candidates_per_query": st["candidates"] / half,
                         "pruning_ratio": 1.0 - st["candidates"] / half / n,
                         "dense_queries": st["dense_queries"],
                         "plain_queries_per_s": 500 / (pms * 1e-3),
                         "plain_candidates_per_query": pst["candidates"] / 500,
                         "identical_answers": bool(torch.equal(ri, ref[0]))}
        groups.append(rec)
    line = {"metric": "learned seed vs descent seed, exact 1-NN at %dx256" % n, "data": "synthetic",
            "config": {"workload": f"{n}x256 random walks; {m} training pairs sigma ~ U[0.1, 1.0]; "
                                   f"{args.study_heldout} held-out queries at sigma 0.1 and 1.0"},
            "generate_s": gen_s, "label_s": label_s, "train_s": train_s, "epochs": args.study_epochs,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]), "by_sigma": groups}
    md.free()
    idx.free()
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import synth
    from oracle import knn as oknn
    n, length = args.n, args.len
    host = synth.random_walk(n, length, seed=1)
    q, _, _ = synth.sigma_queries(host, n, length, args.per_sigma, SIGMAS)
    per = args.per_sigma
    sample_q = q[[0, per, 2 * per]]
    # each step: the three sample queries over a row prefix sized to a few seconds of CPU work
    probe = min(n, 1 << 19)
    t0 = time.perf_counter()
    oknn.knn_chunked(lambda a, b: host[a:b], probe, sample_q, 1)
    tp = time.perf_counter() - t0
    rows = int(min(n, max(probe, probe * 8.0 / max(tp, 1e-3))))
    for _ in range(args.warmup):
        oknn.knn_chunked(lambda a, b: host[a:b], rows, sample_q[:1], 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oknn.knn_chunked(lambda a, b: host[a:b], rows, sample_q, 1)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    qps = len(sample_q) * args.steps / (t * n / rows)
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps * n / rows,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"exact 1-NN over {n}x{length} random-walk fp32 series, w=16, 8-bit iSAX, "
                                   f"queries sigma in {list(SIGMAS)}", "n": n, "len": length},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"3 queries (one per sigma) per step over the first {rows} of {n} rows; "
                                       f"time scaled by {n / rows:.3g} to the full collection"},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bind_local_cpus(dev_index):
    """Runs this process on the CPUs next to the GPU, so that its host buffers (first touched here)
    sit in the memory the GPU's link reaches directly; returns the CPU count or None."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
            return len(cpus)
    except (OSError, ValueError, AttributeError):
        pass
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.learned_study:
        run_learned_study(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    local_cpus = bind_local_cpus(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import paper_2009_00166_gb300 as P
    from paper_2009_00166_gb300 import _build
    if not os.path.exists(P.binding.LIB_PATH):
        _build.build()
    n, length, k = args.n, args.len, args.k
    mode = P.PARIS_MODE_BATCHED if args.mode == "batched" else P.PARIS_MODE_PLAIN
    precision = P.PARIS_REFINE_MIXED if args.precision == "mixed" else P.PARIS_REFINE_FP32
    seed_mode = P.PARIS_SEED_LEARNED if args.seed == "learned" else P.PARIS_SEED_DESCENT
    host, qhost, sig, _ = make_workload(n, length, args.per_sigma, rank)
    X = host.to(dev)
    Q = qhost.to(dev)
    groups = [Q[i * args.per_sigma:(i + 1) * args.per_sigma] for i in range(len(SIGMAS))]
    nq = Q.shape[0]
    stream = torch.cuda.current_stream()

    # ---- learned best-so-far proposal, trained on (query PAA, bucket of its exact nearest
    # neighbour) pairs that the exact method itself labels: before the timed region when the
    # headline uses it, after it otherwise (so that its calls leave no state behind, such as
    # the query tile the library tunes on its first batched call)
    model, training = None, None
    want_model = seed_mode == P.PARIS_SEED_LEARNED or (not args.no_learned_comparison and args.plain_steps > 0)

    def train_model():
        import synth
        t0 = time.perf_counter()
        tq_np, _, _ = synth.mixed_sigma_queries(host.numpy(), n, length, args.train_queries, 0.1, 1.0, seed=20)
        tq = torch.from_numpy(tq_np).to(dev)
        idx = P.paris_build(X, 16, 256)
        nn_rows, _ = P.paris_exact_knn_ex(idx, tq, 1, mode=mode, precision=precision)
        labels = P.paris_row_buckets(idx, nn_rows.cpu().numpy()[:, 0])
        idx.free()
        _, _, tpaa = P.paris_encode(tq, 16, 256, want_paa=True)
        t1 = time.perf_counter()
        md = P.SeedModel(1)
        losses = md.train(tpaa, torch.from_numpy(labels).to(dev), batch=512, epochs=args.train_epochs, lr=2e-3,
                          order_seed=2)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return md, {"pairs": args.train_queries, "label_s": t1 - t0, "train_s": t2 - t1,
                    "epochs": args.train_epochs, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                    "top_r": 3}

    if want_model and seed_mode == P.PARIS_SEED_LEARNED:
        model, training = train_model()

    def step(collect=None, md=mode, prec=precision, sd=seed_mode, answers=None, split=False, prune=True):
        """Build, then answer every query: one call for the whole batch, or one per sigma group."""
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        idx = P.paris_build_ex(X, 16, 256, bf16_shadow=prec == P.PARIS_REFINE_MIXED, leaf_capacity=args.leaf_capacity)
        e1.record(stream)
        if sd == P.PARIS_SEED_LEARNED:
            P.paris_attach_seed_model(idx, model, 3)
        per_sigma_stats = []
        for g in (groups if split else [Q]):
            out = P.paris_exact_knn_ex(idx, g, k, mode=md, precision=prec, seed=sd, want_stats=collect is not None,
                                       query_tile=args.query_tile if md == P.PARIS_MODE_BATCHED else 0,
                                       leaf_pruning=prune)
            if collect is not None:
                per_sigma_stats.append(out[2])
            if answers is not None:
                answers.append(out[0])
        e2.record(stream)
        e2.synchronize()
        idx.free()
        if collect is not None:
            collect.append({"build_ms": e0.elapsed_time(e1), "query_ms": e1.elapsed_time(e2),
                            "stats": per_sigma_stats})
        return e0.elapsed_time(e2)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local, args.clocks_csv)
    launches0 = P.paris_kernel_launches()
    recs = []
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(recs)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    launches = P.paris_kernel_launches() - launches0
    clk = clocks.stop()
    from paper_2009_00166_gb300 import shards
    job_rate, total_ms = shards.job_throughput(total_ms, float(nq * args.steps))

    # ---- end to end through the C ABI with host buffers (copies inside the timed region), right
    # after the device-resident steps and before the comparisons beside them
    e2e = None
    if args.e2e_steps > 0:
        out_i = torch.empty((nq, k), dtype=torch.int64, pin_memory=True)
        out_d = torch.empty((nq, k), dtype=torch.float32, pin_memory=True)
        hq = qhost.numpy()
        times, parts = [], []
        for it in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # host series: copied in by the library
            idx = P.paris_build_ex(host, 16, 256, bf16_shadow=precision == P.PARIS_REFINE_MIXED)
            if seed_mode == P.PARIS_SEED_LEARNED:
                P.paris_attach_seed_model(idx, model, 3)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            P.paris_exact_knn_ex(idx, qhost, k, out_idx=out_i, out_dist=out_d, mode=mode, precision=precision,
                                 seed=seed_mode)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            parts.append((1e3 * (t1 - t0), 1e3 * (times[-1] - (t1 - t0))))
            idx.free()
        # the first pass warms the allocator; the host link is shared with the machine's other
        # jobs, so the steady rate is the median step (the mean is reported beside it)
        steady = sorted(times[1:])
        t_med = steady[len(steady) // 2] if len(steady) % 2 else 0.5 * (steady[len(steady) // 2 - 1] +
                                                                         steady[len(steady) // 2])
        t = t_med * args.e2e_steps
        # the host link's copy rate, beside it (plain copy of the series, not part of the number)
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        X.copy_(host, non_blocking=True)
        torch.cuda.synchronize()
        h2d_gbs = host.numel() * 4 / (time.perf_counter() - c0) / 1e9
        e2e = {"value": nq * args.e2e_steps * world / t, "unit": "queries/s",
               "h2d_bytes_per_step": int(host.numel() * 4 + hq.size * 4),
               "d2h_bytes_per_step": int(nq * k * 12), "h2d_copy_gbs": h2d_gbs, "host_cpus_bound": local_cpus,
               "build_query_ms_per_step": [[round(a, 2), round(b, 2)] for a, b in parts[1:]],
               "mean_value": nq * args.e2e_steps * world / sum(times[1:]), "statistic": "median step"}
        del hq

    # ---- beside it: the plain method (one query per lower-bound pass, fp32 refinement) with the
    # descent seed and with the learned seed, and the headline form per sigma group; answers of
    # every form are compared with the headline's
    def summarize(rs, label):
        ms = [r["build_ms"] + r["query_ms"] for r in rs]
        by = []
        for i, s_ in enumerate(SIGMAS):
            tq = sum(st_["ms_prep"] + st_["ms_descent"] + st_["ms_lbscan"] + st_["ms_refine"] + st_["ms_select"] +
                     st_["ms_dense"] for r in rs for st_ in [r["stats"][i]])
            c = sum(r["stats"][i]["candidates"] for r in rs) / (len(rs) * args.per_sigma)
            pk = sum(r["stats"][i]["pages_kept"] for r in rs) / (len(rs) * args.per_sigma)
            pe = sum(r["stats"][i]["pages_examined"] for r in rs) / (len(rs) * args.per_sigma)
            # summary bytes a query's scans must read: kept pages' summaries plus every page's
            # envelope with leaf pruning, the whole summary array without
            scan_bytes = pk * 256 * 16 + pe * 32 if pe else 16.0 * n
            by.append({"sigma": s_, "queries_per_s": args.per_sigma * len(rs) / (tq * 1e-3),
                       "candidates_per_query": c, "pruning_ratio": 1.0 - c / n,
                       "pages_kept_per_query": pk, "page_keep_ratio": pk / pe if pe else None,
                       "summary_bytes_per_query": scan_bytes,
                       "dense_queries": sum(r["stats"][i]["dense_queries"] for r in rs) / len(rs),
                       "lbscan_ms": sum(r["stats"][i]["ms_lbscan"] for r in rs) / len(rs)})
        return {"form": label, "value": nq * len(rs) / (sum(ms) * 1e-3), "unit": "queries/s",
                "ms_per_step": sum(ms) / len(rs), "by_sigma": by}

    beside, plain_recs, per_sigma = {}, [], None
    if want_model and model is None:
        model, training = train_model()
    if args.plain_steps > 0:
        ans_ref = []
        step(answers=ans_ref)
        forms = [("plain_descent", dict(md=P.PARIS_MODE_PLAIN, prec=P.PARIS_REFINE_FP32, sd=P.PARIS_SEED_DESCENT)),
                 ("plain_no_leaf_pruning", dict(md=P.PARIS_MODE_PLAIN, prec=P.PARIS_REFINE_FP32,
                                                sd=P.PARIS_SEED_DESCENT, prune=False))]
        if model is not None:
            forms.append(("plain_learned", dict(md=P.PARIS_MODE_PLAIN, prec=P.PARIS_REFINE_FP32,
                                                sd=P.PARIS_SEED_LEARNED)))
            forms.append(("headline_learned", dict(sd=P.PARIS_SEED_LEARNED)))
        forms.append(("headline_by_sigma", dict()))
        forms.append(("headline_by_sigma_no_leaf_pruning", dict(prune=False)))
        for name, kw in forms:
            ans = []
            step(answers=ans, split=True, **kw)
            same = bool(torch.equal(torch.cat(ans), ans_ref[0]))
            rs = []
            for _ in range(args.plain_steps):
                step(collect=rs, split=True, **kw)
            beside[name] = summarize(rs, name)
            beside[name]["identical_answers"] = same
            if name == "plain_no_leaf_pruning":
                plain_recs = rs
            if name == "headline_by_sigma":
                per_sigma = beside[name]["by_sigma"]

    # ---- the same batch as a captured plan (one CUDA graph per batch) on an index built once:
    # queries only, replays after the eager first run
    if args.graph_steps > 0:
        idx = P.paris_build_ex(X, 16, 256, bf16_shadow=precision == P.PARIS_REFINE_MIXED)
        plan = P.KnnPlan(idx, nq, k, mode=mode, precision=precision)
        ref_i = P.paris_exact_knn_ex(idx, Q, k, mode=mode, precision=precision)[0]
        gi, _ = plan.run(Q)                                           # eager, then recorded
        for _ in range(2):
            gi, _ = plan.run(Q)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = P.paris_kernel_launches()
        g0.record(stream)
        for _ in range(args.graph_steps):
            gi, _ = plan.run(Q)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.graph_steps
        info = plan.info()
        beside["graph_replay"] = {"form": "captured plan, index built once (queries only)",
                                  "value": nq / (gms * 1e-3), "unit": "queries/s", "ms_per_batch": gms,
                                  "graph_kernels": info["graph_kernels"],
                                  "kernels_per_batch": (P.paris_kernel_launches() - l0) / args.graph_steps,
                                  "eager_runs": info["eager_runs"], "replays": info["replays"],
                                  "identical_answers": bool(torch.equal(gi, ref_i))}
        plan.free()
        idx.free()

    # ---- beside it: the approximate search on adaptive-split ADS+ leaves (a leaf over capacity
    # splits on its most balanced segment) against the fixed-order trie, on an index built once:
    # tree build time and size, seed quality per sigma (seed distance over the true k-th
    # distance), candidates, and queries/s of the headline form with either seed
    if not args.no_adaptive:
        aidx = P.paris_build_ex(X, 16, 256, bf16_shadow=precision == P.PARIS_REFINE_MIXED)
        P.paris_build_adaptive_leaves(aidx)                           # warm-up build
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        P.paris_build_adaptive_leaves(aidx)
        a1.record(stream)
        torch.cuda.synchronize()
        arec = {"form": "ADS+ adaptive-split leaves vs the fixed-order trie (index built once; queries only)",
                "tree_build_ms": a0.elapsed_time(a1), "tree": P.paris_adaptive_leaves_info(aidx)}
        answers = {}
        for name, sd in (("descent", P.PARIS_SEED_DESCENT), ("adaptive", P.PARIS_SEED_ADAPTIVE)):
            _, seed_sq = P.paris_approx_search(aidx, Q, k, seed_mode=sd)
            P.paris_exact_knn_ex(aidx, Q, k, mode=mode, precision=precision, seed=sd)
            ms_, (ai_, ad_, ast_) = timed(lambda: P.paris_exact_knn_ex(aidx, Q, k, mode=mode, precision=precision,
                                                                        seed=sd, want_stats=True), stream, 2)
            answers[name] = ai_
            ratio = (seed_sq.sqrt() / ad_[:, -1].clamp_min(1e-30)).cpu()
            arec[name] = {"value": nq / (ms_ * 1e-3), "unit": "queries/s", "candidates_per_query":
                          ast_["candidates"] / nq, "leaf_rows_per_query": ast_["leaf_rows"] / nq,
                          "dense_queries": ast_["dense_queries"],
                          "seed_over_true_by_sigma": [
                              {"sigma": s_, "mean": float(ratio[i * args.per_sigma:(i + 1) * args.per_sigma].mean()),
                               "median": float(ratio[i * args.per_sigma:(i + 1) * args.per_sigma].median())}
                              for i, s_ in enumerate(SIGMAS)]}
        arec["identical_answers"] = bool(torch.equal(answers["descent"], answers["adaptive"]))
        beside["adaptive_leaves"] = arec
        aidx.free()

    # ---- beside it: the 4096-query batch workload and the three-collection call
    batch_wl = multi_wl = None
    if args.batch_n > 0:
        batch_wl = run_batch_workload(args, P, host, model, dev, stream)
    if args.multi_scale > 0:
        multi_wl = run_three_collections(args, P, dev, stream)

    # ---- beside it: best-so-far sharing ablation (nb-ParIS+ keeps one BSF per worker): the plain
    # method on 300 sigma = 0.1 queries and 100 independent random walks (the hard queries), with
    # the shared BSF and with a private BSF per refining warp
    if args.plain_steps > 0:
        import synth as _synth
        nbq = {"sigma_0.1": Q[args.per_sigma:args.per_sigma + min(300, args.per_sigma)],
               "random_walks": torch.from_numpy(_synth.random_walk(100, length, seed=2)).to(dev)}
        nidx = P.paris_build(X, 16, 256)
        abl = {}
        for gname, gq in nbq.items():
            rec = {}
            ans = {}
            for priv in (False, True):
                _, (gi_, _, st_) = timed(lambda: P.paris_exact_knn_ex(nidx, gq, k, mode=P.PARIS_MODE_PLAIN,
                                                                        want_stats=True, private_bsf=priv), stream, 1)
                rec["private" if priv else "shared"] = {
                    "refined_rows_per_query": st_["refined"] / gq.shape[0],
                    "bsf_updates_per_query": st_["bsf_updates"] / gq.shape[0],
                    "refine_ms": st_["ms_refine"], "queries": int(gq.shape[0])}
                ans[priv] = gi_
            rec["identical_answers"] = bool(torch.equal(ans[False], ans[True]))
            abl[gname] = rec
        beside["nb_ablation"] = abl
        nidx.free()

    # ---- beside it: the same collection kept in host memory (series_on_host): built through two
    # device staging buffers, raw rows read from host memory by the searches; queries only
    if args.graph_steps > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hidx = P.paris_build_ex(host, 16, 256, bf16_shadow=precision == P.PARIS_REFINE_MIXED, series_on_host=True)
        e1.record(stream)
        torch.cuda.synchronize()
        hb_ms = e0.elapsed_time(e1)
        ref_i = P.paris_exact_knn_ex(hidx, Q, k, mode=mode, precision=precision)[0]
        hq_ms, (hi_, _) = timed(lambda: P.paris_exact_knn_ex(hidx, Q, k, mode=mode, precision=precision), stream, 2)
        didx = P.paris_build_ex(X, 16, 256, bf16_shadow=precision == P.PARIS_REFINE_MIXED)
        dq_ms, (di_, _) = timed(lambda: P.paris_exact_knn_ex(didx, Q, k, mode=mode, precision=precision), stream, 2)
        beside["host_resident_series"] = {
            "form": "series kept in host memory, read over the CPU-GPU link (index built once; queries only)",
            "build_ms": hb_ms, "value": nq / (hq_ms * 1e-3), "unit": "queries/s",
            "device_series_value": nq / (dq_ms * 1e-3),
            "identical_answers": bool(torch.equal(hi_, di_)) and bool(torch.equal(ref_i, di_))}
        hidx.free()
        didx.free()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel, from the per-phase device times of the timed steps
    hbm_peak, peak_kind = measured_peaks()
    steps = len(recs)
    ph = {"prep": 0.0, "descent": 0.0, "lbscan": 0.0, "refine": 0.0, "select": 0.0, "dense": 0.0}
    cands = refined = leaf_rows = dense_q = 0
    for r in recs:
        for s in r["stats"]:
            for key in ph:
                ph[key] += s["ms_" + key]
            cands += s["candidates"]
            refined += s["refined"]
            leaf_rows += s["leaf_rows"]
            dense_q += s["dense_queries"]
    build_ms = sum(r["build_ms"] for r in recs) / steps
    query_ms = sum(r["query_ms"] for r in recs) / steps
    # LB-scan roofline (the paper's scan: one query per pass over every summary) from complete
    # single-query scans: the sigma = 0.01 group of the plain-method steps without leaf pruning
    lb_src = plain_recs
    lb_gbs = lb_launch_ms = lb_bytes = None
    if lb_src:
        launches_lb = args.per_sigma * len(lb_src)
        lb_ms0 = sum(r["stats"][0]["ms_lbscan"] for r in lb_src)
        cands0 = sum(r["stats"][0]["candidates"] for r in lb_src)
        lb_bytes = 16.0 * n + 8.0 * cands0 / launches_lb
        lb_launch_ms = lb_ms0 / launches_lb
        lb_gbs = lb_bytes / (lb_launch_ms * 1e-3) / 1e9
    refine_bytes_total = refined * (length * 4.0) + cands * 12.0
    refine_gbs = refine_bytes_total / (ph["refine"] * 1e-3) / 1e9 if ph["refine"] > 0 else 0.0
    dominant = max(ph, key=ph.get)
    wl = {"n": n, "len": length, "queries": nq}    # committed DRAM counters hold only at their own sizes
    if dominant == "dense":
        # algorithmic work of the BF16 screening: 2*len flops per (query, row) pair in the
        # emission pass over every row tile, plus the threshold pass over one row tile in 16; the
        # time is the screening phase's (both passes and their small selection kernels)
        flops = 2.0 * length * n * dense_q * (1.0 + 1.0 / 16.0)
        tf = flops / (ph["dense"] * 1e-3) / 1e12
        peak_tf = bf16_peak_sustained()
        roof = {"kernel": "emit_kernel", "bound": "tensor", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": tf / peak_tf, "traffic": traffic_for("emit_kernel", 0, wl),
                "note": "time of the screening phase: threshold pass (emit_kernel<1>) + emission pass "
                        "(emit_kernel<2>) + selection; traffic is the emission pass's DRAM bytes per launch"}
    elif dominant == "refine":
        roof = {"kernel": "refine_kernel", "bound": "hbm", "achieved": refine_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": refine_gbs / hbm_peak, "traffic": traffic_for("refine_kernel", 0, wl)}
    elif args.mode == "batched":
        # the batched scan is bound by shared-memory table lookups: one 32-bit lookup per lane,
        # slot and query pair, counted by the library (early-abandoned slots are not looked up);
        # peak = 32 banks x 152 SMs x the median SM clock under load
        # (the work-list scan of the queries that keep few pages: 16 lookups per row it tests)
        tile_lookups = float(sum(s["lb_lookups"] for r in recs for s in r["stats"]))
        list_lookups = 16.0 * float(sum(s["list_rows"] for r in recs for s in r["stats"]))
        lookups = tile_lookups + list_lookups
        qt_used = recs[0]["stats"][0]["query_tile"]
        ach = lookups / (ph["lbscan"] * 1e-3) / 1e9
        clk_mhz = clk.get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_l = 32.0 * sms * clk_mhz * 1e6 / 1e9
        kname = "lbscan_batched_kernel" if tile_lookups >= list_lookups else "lbscan_list_kernel"
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": peak_l,
                "unit": "G shared-memory lookups/s", "frac": ach / peak_l,
                "traffic": traffic_for(kname, qt_used if kname == "lbscan_batched_kernel" else 0, wl),
                "lookups_per_step": lookups / steps, "list_lookups_per_step": list_lookups / steps,
                "query_tile": qt_used,
                "summaries_read_per_step_gb_at_most": 16.0 * n * (-(-nq // max(1, qt_used))) / 1e9,
                "note": "time of the whole lower-bound phase (page pass, pilot, ordering, tile and list scans); "
                        "lookups counted on the device"}
    else:
        roof = {"kernel": "lbscan_kernel", "bound": "hbm", "achieved": lb_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": (lb_gbs or 0.0) / hbm_peak, "traffic": traffic_for("lbscan_kernel", 0, wl)}
    roof["peak_kind"] = peak_kind
    value = job_rate
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"build + exact {k}-NN, {n}x{length} random-walk fp32 series (w=16, 8-bit iSAX), "
                               f"{nq} queries = {args.per_sigma} per sigma in {list(SIGMAS)}",
                   "n": n, "len": length, "w": 16, "card": 256, "k": k, "queries_per_step": nq, "mode": args.mode,
                   "l2": f"inputs larger than L2 ({n * length * 4 / 1e9:.1f} GB series; "
                         f"{n * 16 / 1e6:.0f} MB summaries read per query tile)",
                   "parallelism": f"replicas x{world} (independent collections per GPU)"},
        "roofline": roof,
        "lb_scan": None if lb_gbs is None else {
            "achieved_gbs": lb_gbs, "frac_of_hbm": lb_gbs / hbm_peak, "peak_kind": peak_kind,
            "us_per_launch": lb_launch_ms * 1e3, "bytes_per_launch": lb_bytes,
            "launches": "complete one-query scans (sigma=0.01 group of the plain-method steps without leaf pruning)"},
        "lb_scan_frac_of_hbm": None if lb_gbs is None else lb_gbs / hbm_peak,
        "build": {"ms": build_ms, "gb_per_s": n * length * 4 / (build_ms * 1e-3) / 1e9,
                  "series_per_s": n / (build_ms * 1e-3)},
        "query_ms_per_step": query_ms,
        "precision": args.precision,
        "seed": args.seed,
        "seed_training": training,
        "plain_method": beside.get("plain_descent"),
        "beside": beside,
        "dense_queries_per_step": dense_q / steps,
        "phase_ms_per_step": {kk: v / steps for kk, v in ph.items()},
        "per_sigma": per_sigma,
        "batch_50m": batch_wl,
        "three_collections": multi_wl,
        "refine_gbs": refine_gbs,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(host.numpy(), qhost.numpy(), args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
