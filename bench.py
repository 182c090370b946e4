"""Benchmark of the local-mapping search path (correspondence search + map-point fusion).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

A step is one pass of the whole hot path over one batch: the 64 new keyframes of a
64-step EuRoC-shaped batch (5..20 neighbours and 600..2000 keypoints per frame, uneven)
enter the device-resident store (grouping by BoW node + projection grid), then every
(new keyframe, neighbour) pair is searched and every step's map points are fused: one replay
of a CUDA graph of five kernels.  Inputs are synthetic (seeded generator), all
resident in HBM before the timed region; the L2 is flushed (256 MB written) before each
timed step because the batch (~95 MB) fits in L2.  Prints one JSON line.

`e2e` is the same workload through the public batch calls with pinned host buffers: new
keyframes, masks and map points copied in, results copied out, every step; two batches in
flight (the next step's batch begun before the last one's results are taken), and beside it
the one-step-at-a-time call (`e2e.serial`).
The plain one-pair-per-launch form, the oracle on the host cores, and a continuous-batching
serving run (Poisson arrivals) are reported next to it.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcomparisons/s and keyframes/s (search+fuse); p50/p99 per-keyframe latency"
WORKLOAD = "cfg2: 64 independent EuRoC-shaped local-mapping steps, 752x480 f=458, 5-20 neighbours, 600-2000 keypoints/frame"
KP_BYTES = 51     # per stored keypoint read by the path: desc 32, xy 8, angle 4, node 4, orig 2, level 1
MP_BYTES = 65     # per map point: pos 12, normal 12, desc 32, min/max dist 8, skip 1
OUT_BYTES = 12    # per emitted match / fusion candidate
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--serve-kf", type=int, default=3000, help="keyframes of the serving stream (0: skip)")
    ap.add_argument("--serve-kf-20", type=int, default=600,
                    help="keyframes served at 20/s (the stream's first ones; 3000 take 150 s)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-node (tensor-core) workload")
    ap.add_argument("--no-forward", action="store_true", help="skip the step with forward-direction fusion")
    ap.add_argument("--no-configs", action="store_true", help="skip the single-step configurations (cfg0, cfg1, cfg3)")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index  # nvidia-smi -i accepts an index or a GPU UUID
        self.proc = None
        self.lines = []
        self.skip = 0  # readings taken before the timed region

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the first reading marks the start of sampling: the timed region starts after it
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.skip = len(self.lines)
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.skip:] or self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic(kernel_file, profile):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, if the
    kernel source has not changed since the counters were taken."""
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", profile)))
        src = open(os.path.join(ROOT, "paper_2511_02036_gb300", "csrc", kernel_file), "rb").read()
        if prof.get("source_sha256") != hashlib.sha256(src).hexdigest():
            return None, "kernel changed since the ncu capture"
        return prof["dram_bytes_per_launch"], prof.get("note")
    except (OSError, ValueError, KeyError):
        return None, "no ncu capture"


def steps_of(w):
    return [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                 mps=s.get("mps")) for s in w["steps"]]


def algorithmic_bytes(w, res):
    """Unique bytes the path must touch for one batch: every keyframe of the batch once
    (keypoint arrays), the map points once, one mask byte per masked keypoint, 12 bytes per
    output."""
    ids = set()
    mask = 0
    for s in w["steps"]:
        ids.add(s["q"])
        ids.update(s["nbrs"])
        if s.get("q_free") is not None:
            mask += len(s["q_free"])
        if s.get("nbr_free") is not None:
            mask += sum(len(m) for m in s["nbr_free"])
    kp = sum(w["frames"][i]["n"] for i in ids)
    mp = sum(s["mps"]["n"] for s in w["steps"] if s.get("mps") is not None)
    out = len(res.matches) + len(res.fuse)
    return kp * KP_BYTES + mp * MP_BYTES + mask + out * OUT_BYTES, dict(keypoints=kp, map_points=mp,
                                                                         mask_bytes=mask, outputs=out)


def rank_seed(seed, rank):
    """Workload seed of a rank: weak scaling, every rank its own batch of the same shape."""
    return seed + 1000 * rank


def slowest(seconds, dist, device=None):
    """The slowest rank's time (all-reduce MAX over the process group when distributed)."""
    if not dist:
        return float(seconds)
    import torch
    import torch.distributed as D
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world, dist, device=None):
    """Whole-job throughput: the units every rank processed / the slowest rank's time."""
    t = slowest(seconds, dist, device)
    return units_per_rank * world / t, t


def search_bytes(w, res):
    """Algorithmic bytes of the search kernel for one batch: 52 B per keypoint of every query
    and neighbour keyframe (desc 32, xy 8, angle 4, node 4, level 1, caller index 2, mask 1),
    each keyframe once, plus 12 B per output match.  The kernel's own tables (bucket table,
    eligible lists) are implementation, not algorithmic bytes."""
    qs, ts = set(), set()
    for s in w["steps"]:
        qs.add(s["q"])
        ts.update(s["nbrs"])
    q = sum(w["frames"][i]["n"] for i in qs)
    t = sum(w["frames"][i]["n"] for i in ts)
    return 52 * (q + t) + OUT_BYTES * len(res.matches), dict(
        query_keypoints=q, neighbour_keypoints=t, neighbours=len(ts), matches=len(res.matches),
        bytes_per_keypoint=52, bytes_per_match=OUT_BYTES)


def oracle_sample(w, seconds, t_limit=None):
    """The oracle as it stands, single thread, over the workload's steps in order until
    `seconds` of CPU work: returns (keyframes, comparisons, elapsed)."""
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    n = cmp = 0
    k = 0
    while True:
        st = w["steps"][k % len(w["steps"])]
        _, c1 = O.search_step(w["cam"], w["frames"], st)
        _, c2 = O.fuse_step(w["cam"], w["frames"], st)
        n += 1
        cmp += c1 + c2
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds or (t_limit and k >= t_limit):
            return n, cmp, el


def oracle_sample_threads(w, seconds, threads):
    """The same oracle calls on `threads` host threads at once (independent steps, thread i
    taking steps i, i + threads, ...; ctypes releases the GIL inside the oracle's C, which
    keeps no global state) until `seconds` have passed: returns (keyframes, comparisons,
    elapsed).  The oracle's code is unchanged; only independent steps run side by side."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    O.build()
    t0 = time.perf_counter()

    def worker(i):
        n = cmp = 0
        k = i
        while time.perf_counter() - t0 < seconds:
            st = w["steps"][k % len(w["steps"])]
            _, c1 = O.search_step(w["cam"], w["frames"], st)
            _, c2 = O.fuse_step(w["cam"], w["frames"], st)
            n += 1
            cmp += c1 + c2
            k += threads
        return n, cmp

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(worker, range(threads)))
    return sum(r[0] for r in res), sum(r[1] for r in res), time.perf_counter() - t0


# --------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    from gen import workloads as W
    import oracle as O
    w = W.make_cfg2(seed=args.seed)
    # local-mapping steps (keyframes) per timed step: a bounded sample of the batch, about 800
    # oracle steps in all (half a minute on one core) whatever K is, and at least one per step
    per = max(1, min(4, 800 // max(1, args.steps)))
    for _ in range(args.warmup):
        oracle_sample(w, 0.0, t_limit=1)
    t0 = time.perf_counter()
    n = cmp = 0
    k = 0
    for _ in range(args.steps):
        for _ in range(per):
            st = w["steps"][k % len(w["steps"])]
            _, c1 = O.search_step(w["cam"], w["frames"], st)
            _, c2 = O.fuse_step(w["cam"], w["frames"], st)
            cmp += c1 + c2
            n += 1
            k += 1
    el = time.perf_counter() - t0
    kfps = n / el
    line = {"impl": "reference", "metric": METRIC, "value": kfps, "unit": "keyframes/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "%d local-mapping steps per timed step" % per},
            "gcomparisons_per_s": cmp / el / 1e9,
            "cpu_baseline": {"value": kfps, "unit": "keyframes/s", "cores": 1, "kind": "oracle",
                             "sample": "%d steps of the cfg2 batch in order, single thread" % n},
            "e2e": {"value": kfps, "unit": "keyframes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- my arm

def run_mine(args, rank, world, local_rank):
    import torch

    import paper_2511_02036_gb300 as tm
    from gen import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # a stream of our own: the legacy default stream has handle 0, which the library reads
    # as "use the context's stream"
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    dist = world > 1
    if dist:
        import torch.distributed as D

    w = W.make_cfg2(seed=rank_seed(args.seed, rank))  # weak scaling: each rank its own batch
    steps = steps_of(w)
    new_ids = [s["q"] for s in w["steps"]]
    old_ids = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
    ctx = tm.Context(w["cam"], max_kp=2048, device=local_rank)
    ctx.add_keyframes(old_ids, [w["frames"][i] for i in old_ids])

    # device-resident inputs
    st_arr, masks, mps, _keep = tm.pack_batch(steps, ctx.sizes)
    dt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_masks = dt(masks)
    d_mps = {k: (dt(v) if isinstance(v, np.ndarray) else v) for k, v in mps.items()}
    d_new = [dict(desc=dt(f["desc"]), xy=dt(f["xy"]), angle=dt(f["angle"]), level=dt(f["level"]),
                  node=dt(f["node"].view(np.int32)), Tcw=f["Tcw"])
             for f in (w["frames"][i] for i in new_ids)]
    off_steps = [dict(kf_id=st_arr[k].kf_id, nbrs=steps[k]["nbrs"], q_free_off=st_arr[k].q_free_off,
                      nbr_free_off=st_arr[k].nbr_free_off, mp_begin=st_arr[k].mp_begin,
                      mp_count=st_arr[k].mp_count) for k in range(len(steps))]
    torch.cuda.synchronize(dev)
    plan = ctx.plan(off_steps, masks=d_masks, mps=d_mps, new=(new_ids, d_new))
    info = plan.info()
    tuning = plan.tuning()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist:
            D.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        plan.run(stream)
    torch.cuda.synchronize(dev)
    res = plan.results(stream)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = []
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = Clocks(("GPU-%s" % uuid) if uuid is not None else local_rank)
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        plan.run(stream)
        ev1[k].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    # stage times (the match kernel's among them) from the plan's timed graph, which records
    # CUDA events on the launching stream at the stage boundaries, same inputs, L2 flushed
    for k in range(args.steps):
        flush.zero_()
        plan.run(stream, timed=True)
        stage.append(plan.stage_times())  # waits for this run
    stage = np.array(stage)
    # warm L2: the same replays back to back without the flush (the batch fits in L2)
    for k in range(args.steps):
        ev0[k].record(stream)
        plan.run(stream)
        ev1[k].record(stream)
    torch.cuda.synchronize(dev)
    warm = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    value, total_s = job_throughput(len(new_ids) * args.steps, step_ms.sum() / 1e3, world, dist, dev)
    res2 = plan.results(stream)
    assert np.array_equal(res.matches, res2.matches) and np.array_equal(res.fuse, res2.fuse)
    ncmp = res.n_comparisons_search + res.n_comparisons_fuse
    gcomp = ncmp * args.steps * world / total_s / 1e9

    # roofline of the dominant kernel (match), timed by the events around it in the timed graph
    pk, pk_kind = peaks()
    alg, parts = search_bytes(w, res)
    path_bytes, path_parts = algorithmic_bytes(w, res)
    kern_ms = float(stage[:, 0].mean())
    achieved = alg / (kern_ms / 1e3) / 1e9
    traffic, traffic_note = kernel_traffic("kernels.cu", "search_kernel_cfg2.json")
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "kernel": "search_kernel (CTA per pair: F, node join, Hamming/epipolar search, one match per target, rotation filter, compaction)",
            "peak_kind": pk_kind, "algorithmic_bytes": alg, "algorithmic_parts": parts,
            "kernel_ms": kern_ms, "traffic_note": traffic_note,
            "path_algorithmic_bytes": path_bytes, "path_parts": path_parts}
    roof["path_frac"] = (path_bytes / (float(step_ms.mean()) / 1e3) / 1e9) / pk["hbm_gbs"]
    roof["path_note"] = ("path_frac: the whole step's algorithmic bytes (every keyframe, map point, "
                         "mask byte and output once) / ms_per_step / the HBM peak")
    # the ALU side: per comparison 8 XOR + 8 POPC (a 256-bit Hamming distance); peak rates
    # measured on this device by the library's probe kernel (tm_measure_int_rates)
    rates = tm.int_rates(local_rank)
    t_alu = max(8 * res.n_comparisons_search / rates["popc_per_s"],
                res.n_comparisons_search / rates["hamming_per_s"])
    t_hbm = alg / (pk["hbm_gbs"] * 1e9)
    roof["alu_check"] = {"popc_per_comparison": 8, "comparisons": int(res.n_comparisons_search),
                         "popc_per_s": rates["popc_per_s"], "lop3_per_s": rates["lop3_per_s"],
                         "hamming_per_s": rates["hamming_per_s"], "rates": "measured (probe kernel, best of 3)",
                         "t_alu_us": 1e6 * t_alu, "t_hbm_us": 1e6 * t_hbm,
                         "t_roof_us": 1e6 * max(t_alu, t_hbm), "frac_of_t_roof": max(t_alu, t_hbm) / (kern_ms / 1e3),
                         "note": "T_roof = max(bytes / HBM peak, comparisons x 8 / POPC rate, comparisons / "
                                 "Hamming rate); the HBM term binds"}

    out = {"metric": METRIC, "value": value, "unit": "keyframes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(step_ms.mean()),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32",
           "data": "synthetic (seeded generator; EuRoC-shaped)",
           "config": {"workload": WORKLOAD, "new_keyframes_per_step": len(new_ids),
                      "pairs": sum(len(s["nbrs"]) for s in steps), "map_points": int(mps["n"]),
                      "l2": "flushed before each timed step (256 MB written)",
                      "launch": dict(info, tuning=tuning), "parallelism": "replicas" if world == 1 else "dp%d" % world},
           "gcomparisons_per_s": gcomp,
           "comparisons_per_step": ncmp,
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                          "note": "batch form: every keyframe of a step completes with its batch"},
           "stage_ms": {"search": kern_ms, "ingest": float(stage[:, 1].mean()),
                        "fuse": float(stage[:, 2].mean()), "copy": float(stage[:, 3].mean()),
                        "note": "from the plan's timed graph (an event node at each stage boundary "
                                "adds a few us); the search kernel runs beside the store branch "
                                "(ingest, then fuse); copy = from the later of the search and fusion "
                                "kernels' ends to the end of the run (each branch compacts its own "
                                "records); value and ms_per_step come from the kernels-only graph"},
           "warm_l2": {"ms_per_step": float(warm.mean()), "value": len(new_ids) / (float(warm.mean()) / 1e3),
                       "unit": "keyframes/s", "note": "same replays back to back without the L2 flush"},
           "device": torch.cuda.get_device_name(dev), "roofline": roof, "clocks": clk, "gpu_launches": int(info["kernels_per_run"]) * args.steps,
           "wall_s_timed_region": t_wall}

    # ---------------------------------------------------------------- plain per-pair form
    if not args.no_plain:
        pplan = None
        try:
            pplan = ctx.plan(off_steps, masks=d_masks, mps=d_mps, sp=tm.SearchParams(mode=tm.TM_MODE_PER_PAIR))
            pplan.run(stream)
            torch.cuda.synchronize(dev)
            pres = pplan.results(stream)
            assert np.array_equal(pres.matches, res.matches) and np.array_equal(pres.fuse, res.fuse)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0.record(stream)
                pplan.run(stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            pms = float(np.mean(ms))
            out["plain_form"] = {"value": len(new_ids) / (pms / 1e3), "unit": "keyframes/s",
                                 "ms_per_step": pms, "kernels_per_step": pplan.info()["kernels_per_run"],
                                 "note": "same batch, one pair per launch sequence (memsets + 3 kernels per pair, 2 per fusion), keyframes already stored"}
        finally:
            if pplan is not None:
                pplan.close()

    plan.close()

    # ---------------------------------------------------------------- end to end
    if not args.no_e2e:
        for i in new_ids:
            ctx.remove_keyframe(i)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        h_masks = pin(masks)
        # the map points in one page-locked staging block (uploaded with one copy)
        h_mps = tm.pack_mappoints(mps)
        # the new keyframes packed one after another, one pinned array per field (as a producer
        # streaming keyframes into a staging buffer would hand them over)
        fr = [w["frames"][i] for i in new_ids]
        h_new = dict(n=[f["n"] for f in fr], desc=pin(np.concatenate([f["desc"] for f in fr])),
                     xy=pin(np.concatenate([f["xy"] for f in fr])), angle=pin(np.concatenate([f["angle"] for f in fr])),
                     level=pin(np.concatenate([f["level"] for f in fr])),
                     node=pin(np.concatenate([f["node"] for f in fr]).view(np.int32)),
                     Tcw=np.stack([np.asarray(f["Tcw"], np.float64).reshape(12) for f in fr]))
        # bytes copied in per step: masks, map-point arrays, the new keyframes' arrays
        # (desc 32 + xy 8 + angle 4 + level 1 + node 4 = 49 B per keypoint), the work list (the
        # library's 128-byte work records: every item, and the search's launch entries once
        # more), the new keyframes' ingest records (112 B each) and the gather records of their
        # packed arrays (48 B per 1024 keypoints)
        n_pairs = sum(len(s["nbrs"]) for s in steps)
        n_items = n_pairs + sum((s["mps"]["n"] + 511) // 512 for s in steps)
        n_units = tuning["search_units"]  # launch entries of the search (split pairs twice)
        h2d = (int(masks.nbytes) + int(h_mps["block"].numel())
               + sum(w["frames"][i]["n"] for i in new_ids) * 49
               + (n_items + n_units) * 128 + len(new_ids) * 112
               + 48 * ((sum(w["frames"][i]["n"] for i in new_ids) + 1023) // 1024))
        # out: item offsets, comparison totals (3 x 8 B) and the status word, the results
        d2h = 4 * (n_items + 1) + 24 + 4 + OUT_BYTES * (len(res.matches) + len(res.fuse))

        # the step table as columns (how a producer of batches hands it over; built once here
        # because every timed step runs the same batch)
        table = tm.StepTable.from_steps(off_steps)

        def e2e_step():
            r = ctx.batch_run(table, masks=h_masks, mps=h_mps, new=(new_ids, h_new))
            ctx.remove_keyframes(new_ids)
            return r

        ke = max(3, args.steps // 2)
        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            r = e2e_step()
        barrier()
        serial_value, serial_el = job_throughput(len(new_ids) * ke, time.perf_counter() - t0, world, dist, dev)
        assert np.array_equal(r.matches, res.matches) and np.array_equal(r.fuse, res.fuse)

        # pipelined: the batches of steps k + 1 and k + 2 are begun (marshalled, uploaded,
        # launched) before the results of step k are taken, so that the host prepares while
        # earlier batches transfer and run.  Each batch stores its 64 new keyframes under an id
        # set of its own (16 sets in turn); once 8 batches are finished their keyframes are
        # removed in one call (inside the timed region), so that the store stays bounded and a
        # set is free again before it comes round
        depth, group, nsets = 3, 8, 16
        ids2 = [[i + (j << 40) for i in new_ids] for j in range(nsets)]
        tables = [table] + [tm.StepTable.from_steps([dict(st, kf_id=i) for st, i in zip(off_steps, ids2[j])])
                            for j in range(1, nsets)]

        # results as views into caller-owned pinned buffers, one set per batch in flight
        outs = [tm.ResultBuffers() for _ in range(depth)]

        def retire(k, n, done):
            """After batch k of n is finished: remove the keyframes of the last `group` batches."""
            done.extend(ids2[k % nsets])
            if (k + 1) % group == 0 or k == n - 1:
                ctx.remove_keyframes(done)
                done.clear()

        def pipelined(n):
            inflight, last, done = [], None, []
            for k in range(n + depth - 1):
                if k < n:
                    inflight.append((ctx.batch_begin(tables[k % nsets], masks=h_masks, mps=h_mps,
                                                     new=(ids2[k % nsets], h_new)), k))
                if len(inflight) == depth or (k >= n and inflight):
                    t, kk = inflight.pop(0)
                    last = ctx.batch_finish(t, out=outs[kk % depth])
                    retire(kk, n, done)
            return last

        # the same stream of batches from two host threads: a producer begins them (at most
        # `depth` in flight), a consumer finishes each in order and retires its keyframes, so the
        # binding's marshalling of one batch overlaps the library's work on others
        import queue

        def threaded(n):
            sem, q, err, last, done = threading.Semaphore(depth), queue.Queue(), [], [None], []

            def consumer():
                while True:
                    item = q.get()
                    if item is None:
                        return
                    try:
                        if not err:
                            t, k = item
                            last[0] = ctx.batch_finish(t, out=outs[k % depth])
                            retire(k, n, done)
                    except BaseException as ex:  # noqa: BLE001 (reported by the producer)
                        err.append(ex)
                    sem.release()

            th = threading.Thread(target=consumer, daemon=True)
            th.start()
            try:
                for k in range(n):
                    sem.acquire()
                    if err:
                        break
                    q.put((ctx.batch_begin(tables[k % nsets], masks=h_masks, mps=h_mps,
                                           new=(ids2[k % nsets], h_new)), k))
            finally:
                q.put(None)
                th.join()
            if err:
                raise err[0]
            return last[0]

        pipelined(max(2, args.warmup))
        barrier()
        t0 = time.perf_counter()
        r = pipelined(ke)
        barrier()
        one_value, one_el = job_throughput(len(new_ids) * ke, time.perf_counter() - t0, world, dist, dev)
        assert np.array_equal(r.matches, res.matches) and np.array_equal(r.fuse, res.fuse)
        threaded(max(2, args.warmup))
        barrier()
        t0 = time.perf_counter()
        r = threaded(ke)
        barrier()
        e2e_value, el = job_throughput(len(new_ids) * ke, time.perf_counter() - t0, world, dist, dev)
        assert np.array_equal(r.matches, res.matches) and np.array_equal(r.fuse, res.fuse)
        out["e2e"] = {"value": e2e_value, "unit": "keyframes/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": 1e3 * el / ke,
                      "api": "Context.batch_begin / batch_finish -> tm_batch_begin / tm_batch_finish, three "
                             "batches in flight, begun by a producer thread and finished in order by a consumer "
                             "thread (step table as columns; pinned host buffers: new keyframes, masks, map "
                             "points (one staging block, one copy) in; matches and fusion candidates out, into "
                             "one caller-owned ResultBuffers "
                             "per batch in flight, returned as views) + Context.remove_keyframes of the new "
                             "keyframes of every 8 finished steps in one call (consumer)",
                      "link": "inputs cross the host link at about 205 GB/s on this GB300 (copy engine and SM "
                              "loads alike): ~0.2 ms of the step's 40 MB",
                      "one_thread": {"value": one_value, "unit": "keyframes/s", "ms_per_step": 1e3 * one_el / ke,
                                     "api": "the same three batches in flight from one host thread (steps k + 1 "
                                            "and k + 2 begun before step k's results are taken)"},
                      "serial": {"value": serial_value, "unit": "keyframes/s", "ms_per_step": 1e3 * serial_el / ke,
                                 "api": "Context.batch_run -> tm_batch_run, one step at a time"}}

    # ---------------------------------------------------------------- dense node blocks
    if not args.no_dense and rank == 0:
        out["dense_blocks"] = run_dense(tm, stream, flush, local_rank, max(3, args.steps // 2))

    # ---------------------------------------------------------------- forward fusion
    if not args.no_forward and rank == 0:
        out["forward_fusion"] = run_forward(tm, stream, flush, local_rank, max(3, args.steps // 2), args.seed)

    # ---------------------------------------------------------------- single-step configurations
    if not args.no_configs and rank == 0:
        out["configs"] = run_configs(tm, stream, flush, local_rank, max(20, args.steps), min(2.0, args.cpu_seconds / 4))

    # ---------------------------------------------------------------- serving
    if args.serve_kf > 0 and rank == 0:
        out["serving"] = run_serving(tm, args.serve_kf, local_rank, args.serve_kf_20)

    # ---------------------------------------------------------------- oracle on host cores
    if rank == 0:
        n, cmp, el = oracle_sample(w, args.cpu_seconds)
        out["cpu_baseline"] = {"value": n / el, "unit": "keyframes/s", "cores": 1, "kind": "oracle",
                               "sample": "%d local-mapping steps of the same batch in order (search + fusion), single thread, %.1f s" % (n, el),
                               "gcomparisons_per_s": cmp / el / 1e9}
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        n, cmp, el = oracle_sample_threads(w, args.cpu_seconds / 2, threads)
        out["cpu_baseline"]["all_cores"] = {
            "value": n / el, "unit": "keyframes/s", "cores": threads,
            "sample": "%d steps of the same batch, independent steps on %d threads at once, %.1f s" % (n, threads, el),
            "gcomparisons_per_s": cmp / el / 1e9}
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def dense_comparisons(w, st, dmin):
    """(query, candidate) pairs of a step inside dense node blocks: per pair and node with at
    least dmin neighbour keypoints, eligible queries x eligible neighbour keypoints."""
    Q = w["frames"][st["q"]]
    fq = np.ones(Q["n"], bool) if st.get("q_free") is None else np.asarray(st["q_free"]) != 0
    total = 0
    for k, t in enumerate(st["nbrs"]):
        T = w["frames"][t]
        ft = np.ones(T["n"], bool) if st.get("nbr_free") is None else np.asarray(st["nbr_free"][k]) != 0
        nodes, counts = np.unique(T["node"], return_counts=True)
        for nd in nodes[counts >= dmin]:
            total += int(np.count_nonzero(fq & (Q["node"] == nd))) * int(np.count_nonzero(ft & (T["node"] == nd)))
    return total


def run_dense(tm, stream, flush, device, reps):
    """Dense node blocks on the tensor cores against the candidate rounds, same results
    required: the batched workload (64 TUM-VI-shaped steps of cfg3b's model -- new keyframe +
    20 neighbours, 1500 keypoints, 16 BoW nodes, so ~94 x 94 same-node blocks -- 1280 pairs
    in one plan, search only) and the single cfg3b step."""
    import torch
    from gen import workloads as W
    out = {"dense_min": 64}
    for name, w in (("batched", W.make_cfg3b_batch()), ("single_step", W.make_cfg3b())):
        steps = [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"))
                 for s in w["steps"]]
        row = {"workload": ("64 steps x (new keyframe + 20 neighbours), 512x512 f=190, 1500 keypoints, "
                            "16 BoW nodes, masks; 1280 pairs" if name == "batched" else
                            "cfg3b: one step, new keyframe + 20 neighbours, 1500 keypoints, 16 BoW nodes, masks")}
        with tm.Context(w["cam"], max_kp=2048, device=device) as ctx:
            ids = sorted(set(i for s in w["steps"] for i in [s["q"]] + list(s["nbrs"])))
            ctx.add_keyframes(ids, [w["frames"][i] for i in ids])
            results = {}
            for form, dmin in (("tensor_cores", 64), ("candidate_rounds", 0)):
                with ctx.plan(steps, sp=tm.SearchParams(dense_min=dmin)) as plan:
                    for _ in range(3):
                        plan.run(stream)
                    torch.cuda.synchronize()
                    res = plan.results(stream)
                    ms = time_plan(plan, stream, flush, reps)
                    stage = []
                    for _ in range(reps):
                        flush.zero_()
                        plan.run(stream, timed=True)
                        stage.append(plan.stage_times())
                    stage = np.array(stage).mean(axis=0)
                    results[form] = res
                    row[form] = {"ms_per_step": float(ms.mean()), "keyframes_per_s": len(steps) / (float(ms.mean()) / 1e3),
                                 "gcomparisons_per_s": res.n_comparisons_search / (float(ms.mean()) / 1e3) / 1e9,
                                 "search_kernel_ms": float(stage[0]), "dense_kernel_ms": float(stage[4]),
                                 "kernels_per_run": plan.info()["kernels_per_run"], "tuning": plan.tuning()}
            a, b = results["tensor_cores"], results["candidate_rounds"]
            assert np.array_equal(a.matches, b.matches) and a.n_comparisons_search == b.n_comparisons_search
            ncmp_dense = sum(dense_comparisons(w, st, 64) for st in w["steps"])
            pk, pk_kind = peaks()
            fp8_peak = 2.0 * pk["bf16_tflops"]  # dense fp8 = 2 x bf16 (nominal 4.5 vs 2.25 PFLOP/s)
            dms = row["tensor_cores"]["dense_kernel_ms"]
            flops = 2.0 * 256 * ncmp_dense  # one 256-long +-1 dot product per (query, candidate)
            row["comparisons"] = a.n_comparisons_search
            row["dense_comparisons"] = ncmp_dense
            row["speedup"] = row["candidate_rounds"]["ms_per_step"] / row["tensor_cores"]["ms_per_step"]
            row["roofline"] = {"bound": "tensor", "kernel": "dense_kernel", "achieved": flops / (dms / 1e3) / 1e12,
                               "peak": fp8_peak, "unit": "TFLOP/s", "frac": flops / (dms / 1e3) / 1e12 / fp8_peak,
                               "peak_kind": pk_kind + " bf16 burst x 2 (fp8/bf16 nominal ratio)",
                               "algorithmic_flops": flops, "traffic": None}
        out[name] = row
    return out


def run_forward(tm, stream, flush, device, reps, seed):
    """The cfg2 batch with forward-direction fusion as well (Sec. IV-D: the new keyframes' own
    map points fused into every neighbour, skipping those a neighbour already observes), as one
    plan: step time and the forward work, against the same batch without it."""
    import torch
    from gen import workloads as W
    w = W.make_cfg2(seed=seed, forward=True)
    new_ids = [s["q"] for s in w["steps"]]
    old_ids = sorted(set(i for s in w["steps"] for i in s["nbrs"]))
    out = {"workload": "cfg2 + forward fusion: the same 64 steps; per step its new keyframe's map points "
                       "(mapped and just-triangulated points it observes) into each of its neighbours; "
                       "and the same with every match triangulated and checked on the GPU"}
    with tm.Context(w["cam"], max_kp=2048, device=device) as ctx:
        ctx.add_keyframes(old_ids, [w["frames"][i] for i in old_ids])
        for name, fwd, tri in (("with_forward", True, False), ("without_forward", False, False),
                               ("with_forward_and_triangulation", True, True)):
            steps = [dict(kf_id=s["q"], nbrs=s["nbrs"], q_free=s.get("q_free"), nbr_free=s.get("nbr_free"),
                          mps=s.get("mps"), **({"fwd_mps": s["fwd_mps"], "fwd_skip": s["fwd_skip"]} if fwd else {}))
                     for s in w["steps"]]
            with ctx.plan(steps, new=(new_ids, [w["frames"][i] for i in new_ids]),
                          tri=tm.TriParams() if tri else None) as plan:
                for _ in range(3):
                    plan.run(stream)
                torch.cuda.synchronize()
                res = plan.results(stream)
                e0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
                e1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
                for k in range(reps):
                    flush.zero_()
                    e0[k].record(stream)
                    plan.run(stream)
                    e1[k].record(stream)
                torch.cuda.synchronize()
                ms = float(np.mean([a.elapsed_time(b) for a, b in zip(e0, e1)]))
                out[name] = {"ms_per_step": ms, "keyframes_per_s": len(new_ids) / (ms / 1e3),
                             "kernels_per_run": plan.info()["kernels_per_run"],
                             "forward_candidates": int(len(res.fwd)), "forward_comparisons": int(res.n_comparisons_fwd),
                             "forward_map_points": int(sum(s["fwd_mps"]["n"] * len(s["nbrs"]) for s in w["steps"])) if fwd else 0}
                if tri:
                    out[name]["triangulated_matches"] = int(len(res.matches))
                    out[name]["accepted_new_points"] = int(res.point_ok.sum())
            ctx.remove_keyframes(new_ids)  # the plan's new keyframes stay stored after it
    return out


def time_plan(plan, stream, flush, reps):
    """Device milliseconds of `reps` replays of a plan, each after an L2 flush, timed by
    CUDA events on the launching stream."""
    import torch
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for k in range(reps):
        flush.zero_()
        e0[k].record(stream)
        plan.run(stream)
        e1[k].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in zip(e0, e1)])


def config_workloads():
    """The single-step configurations: (name, description, workload in the step format)."""
    from gen import workloads as W
    p = W.make_pair_cfg0(0)
    cfg0 = dict(cam=p["cam"], frames=[p["Q"], p["T"]], steps=[dict(q=0, nbrs=[1])])
    return [("cfg0", "single pair: 640x480 f=450, 500 keypoints, 200 planted correspondences, "
                     "0.3 m baseline, 5 deg yaw, 1000 BoW nodes, no masks, no fusion", cfg0),
            ("cfg1", "EuRoC-shaped step: 752x480 f=458, new keyframe + 10 neighbours, 1200 keypoints, "
                     "40% shared points, masks, ~6000 map points fused", W.make_cfg1()),
            ("cfg3", "TUM-VI-shaped step: 512x512 f=190, new keyframe + 20 neighbours, 1500 keypoints, "
                     "50% shared, flip 0.08, 10000 BoW nodes, masks, map points fused", W.make_cfg3())]


def run_configs(tm, stream, flush, device, reps, cpu_seconds):
    """cfg0, cfg1 and cfg3, one step each: the fused plan (new keyframe ingested in the step,
    search, fusion: one graph) against the plain per-pair form (neighbours and new keyframe
    already stored), both checked against the oracle element by element, and the oracle on
    one host core and on all of them."""
    import oracle as O
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    out = {}
    for name, desc, w in config_workloads():
        st = w["steps"][0]
        exp_pairs, ecs = O.search_step(w["cam"], w["frames"], st)
        exp_fuse, ecf = O.fuse_step(w["cam"], w["frames"], st)
        steps = [dict(kf_id=st["q"], nbrs=st["nbrs"], q_free=st.get("q_free"), nbr_free=st.get("nbr_free"),
                      mps=st.get("mps"))]
        row = {"workload": desc, "pairs": len(st["nbrs"]), "comparisons_per_step": int(ecs + ecf),
               "map_points": int(st["mps"]["n"]) if st.get("mps") is not None else 0}
        with tm.Context(w["cam"], max_kp=2048, device=device) as ctx:
            ctx.add_keyframes(list(st["nbrs"]), [w["frames"][i] for i in st["nbrs"]])
            for form, kw in (("batched", dict(new=([st["q"]], [w["frames"][st["q"]]]))),
                             ("plain", dict(sp=tm.SearchParams(mode=tm.TM_MODE_PER_PAIR)))):
                with ctx.plan(steps, **kw) as plan:
                    for _ in range(3):
                        plan.run(stream)
                    res = plan.results(stream)
                    # parity with the oracle, element by element, for this form
                    assert len(res.pairs) == len(exp_pairs)
                    for g, e in zip(res.pairs, exp_pairs):
                        assert np.array_equal(g, e), (name, form)
                    assert np.array_equal(res.fuses[0], exp_fuse), (name, form)
                    assert res.n_comparisons_search == ecs and res.n_comparisons_fuse == ecf
                    ms = time_plan(plan, stream, flush, reps)
                    row[form] = {"keyframes_per_s": 1e3 / float(ms.mean()), "ms_per_step": float(ms.mean()),
                                 "gcomparisons_per_s": (ecs + ecf) / (float(ms.mean()) / 1e3) / 1e9,
                                 "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                                 "kernels_per_run": plan.info()["kernels_per_run"], "parity": "oracle, bit-exact"}
        row["batched"]["note"] = "includes the new keyframe's ingest into the store"
        row["plain"]["note"] = "new keyframe already stored; one launch sequence per pair"
        n, cmp, el = oracle_sample(w, cpu_seconds)
        row["oracle_1_core"] = {"keyframes_per_s": n / el, "gcomparisons_per_s": cmp / el / 1e9,
                                "sample": "%d repetitions of the step, %.1f s" % (n, el)}
        n, cmp, el = oracle_sample_threads(w, cpu_seconds, threads)
        row["oracle_all_cores"] = {"keyframes_per_s": n / el, "gcomparisons_per_s": cmp / el / 1e9, "cores": threads,
                                   "sample": "%d repetitions of the step on %d threads, %.1f s" % (n, threads, el)}
        out[name] = row
    return out


def run_serving(tm, n_kf, device, rate20_kf):
    """Continuous batching on the cfg4 stream (n_kf keyframes along a 10-minute trajectory,
    752x480, 1000-2000 keypoints, 5-20 neighbours; store budget 5000 keyframe slots):
    Poisson arrivals at 20, 100 and 500 keyframes/s, every request at once (the served
    ceiling), a tight store (64 slots, the oldest keyframes evicted) at 500/s and at once,
    showing admission by memory, and the plain per-pair form served one request at a time at 500/s
    and at once.  The 20/s rate serves the stream's first rate20_kf keyframes (its full
    length takes n_kf / 20 seconds of wall time)."""
    from gen import workloads as W
    w = W.make_stream_cfg4(seed=4000, n_kf=n_kf, duration_s=600.0 * n_kf / 3000.0)
    out = {"keyframes": n_kf, "stream": "cfg4: 752x480 f=458, 1000-2000 keypoints, 5-20 neighbours, "
                                        "10-minute trajectory, masks, map points fused"}
    with tm.Context(w["cam"], max_kp=2048, device=device) as probe:
        slot = probe.stats()["slot_bytes"]
    out["store_budget"] = {"slots": 5000, "slot_bytes": slot, "bytes": 5000 * slot}

    def serve(rate, n=None, slots=5000, **cfg):
        n = n or n_kf
        rng = np.random.default_rng(7)
        arr = np.cumsum(rng.exponential(1.0 / rate, n)) if rate else np.zeros(n)
        with tm.Context(w["cam"], max_kp=2048, budget=slots * slot, device=device) as ctx:
            ctx.reserve(min(slots, n + 64))  # the store's slots allocated before serving starts
            with ctx.server(**cfg) as srv:
                t0 = time.perf_counter()
                t0_lib = tm.tm_now()
                tickets = []
                for k, st in enumerate(w["steps"][:n]):
                    while time.perf_counter() - t0 < arr[k]:
                        time.sleep(1e-4)
                    tickets.append(srv.submit(st["q"], w["frames"][st["q"]], st["nbrs"], st["q_free"],
                                              st["nbr_free"], st["mps"]))
                lat, done = [], 0.0
                for t in tickets:
                    info = srv.poll(t, timeout=600.0)
                    assert info["done"] and info["status"] == 0
                    lat.append(info["t_done"] - info["t_submit"])
                    done = max(done, info["t_done"])
                    srv.take(t)
                stats = srv.stats()
        lat = np.array(lat) * 1e3
        return {"keyframes": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "offered_kf_per_s": rate if rate else "all at once",
                "served_kf_per_s": n / (done - t0_lib), "server": stats}

    batched = dict(max_batch_requests=64, max_inflight_batches=3)
    out["continuous_batching_20"] = serve(20, n=min(n_kf, rate20_kf), **batched)
    for rate in (100, 500):
        out["continuous_batching_%d" % rate] = serve(rate, **batched)
    out["continuous_batching_all_at_once"] = serve(0, **batched)
    for name, rate in (("continuous_batching_500_tight_store", 500), ("continuous_batching_all_at_once_tight_store", 0)):
        tight = serve(rate, slots=64, evict_after=40, **batched)
        tight["note"] = ("store budget 64 slots, the server keeps the newest 40 of its keyframes: a batch "
                         "takes only the slots that are free, the rest of the queue waits for slots as "
                         "earlier batches retire and their keyframes can be evicted (server.deferrals)")
        out[name] = tight
    plain = dict(max_batch_requests=1, max_inflight_batches=1, sp=tm.SearchParams(mode=tm.TM_MODE_PER_PAIR))
    out["plain_per_pair_500"] = serve(500, **plain)
    out["plain_per_pair_all_at_once"] = serve(0, **plain)
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as D
        torch.cuda.set_device(local_rank)
        D.init_process_group("nccl" if args.impl == "mine" else "gloo")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            import __graft_entry__ as g
            if rank == 0 or world == 1:
                g.build()
            if world > 1:
                import torch.distributed as D
                D.barrier()
                g.build()
            run_mine(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as D
            D.destroy_process_group()


if __name__ == "__main__":
    main()
