"""Benchmark of the 7L online sampler on B300.

One step = one batched call of the online sampler (Algorithm I steps 2-8:
network, Philox normal, g_m, state update, FP64 per-set moments) over the
GBM workload: 16 parameter sets theta=(mu,sigma) ~ U([0,0.2]x[0.1,0.5]),
10^6 paths each, Y0=1, T=2, 16 coarse steps, m=7, network 4->50x4->7 ReLU.
Metric: path-steps/s (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|fp32]
                  [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun (N ranks) the job is one batch
of 16 N parameter sets (10^6 paths each) split across the ranks by path count
(paper_2302_05170_b300.sharding): every rank runs its contiguous range of the
flat path list, and the per-set FP64 partial moments are combined with one
all-gather per step.  Per-GPU work is fixed as N grows: weak scaling.  The
process group is NCCL; SL_DIST_BACKEND=gloo selects gloo (host collectives),
and ranks beyond the visible GPUs share them (LOCAL_RANK modulo the count).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "path-steps/s (7L online, BF16-TC vs FP32) at <=2e-3 rel err; EM label samples/s"
UNIT = "path-steps/s"
WORKLOAD = "GBM 7L online: 16 theta x 1e6 paths x 16 coarse steps, m=7, MLP 4->50x4->7 ReLU"
ALG_FLOPS_PER_PATH_STEP = 2 * (4 * 50 + 3 * 50 * 50 + 50 * 7)   # 16,100 (biases excluded)
# 7L-CDC in the marginal's quantile coordinate, m = 7, per path-step inside the hull: m Horner
# evaluations of degree m - 1 in X and one in xi (FMA = 2 flops); the normal draw is not counted
CDC_FLOPS_PER_PATH_STEP = 2 * 7 * 6 + 2 * 6                            # 96
# network training of the bench (pipeline.train_network keywords): features and labels normalised
# for training, 4e5 Euler-Maruyama paths per label row, and a BF16 finish, so that the FP32 and the
# tensor-core forms evaluate the same (BF16-valued) trained network
TRAIN_RECIPE = dict(normalize=True, n_paths=400_000, bf16_steps=10_000)
# step sizes of the networks used at dt = 1/64 (the adjoint workload: T = 1 in 64 steps)
ADJ_DTS = (1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2, 1.0)


def take(t, idx):
    """Values of a device tensor at the flat indices idx (numpy FP64)."""
    import torch
    return t[torch.as_tensor(idx, device=t.device)].double().cpu().numpy()


def sample_idx(offsets, per_set, seed=12):
    """A bounded sample of flat path indices: per_set paths of every set (its first and last
    included), for the FP64 oracle checks."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(len(offsets) - 1):
        a, b = int(offsets[s]), int(offsets[s + 1])
        if b <= a:
            continue
        k = min(per_set, b - a)
        out.append(np.unique(np.concatenate([[a, b - 1], rng.integers(a, b, k)])))
    return np.concatenate(out) if out else np.zeros(0, np.int64)

# DRAM traffic of the sampler kernel on the default workload, from the committed ncu summary;
# used only while the kernel's sources are those the counters were taken on.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "tc_7l_kernel_gbm_online.md")
KERNEL_SOURCES = ("sl_tc.cu", "sl_tc_common.cuh", "sl_internal.cuh", "sl_fastnormal.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2302_05170_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum), or None when the summary
    is missing or was taken on other kernel sources."""
    try:
        with open(TRAFFIC_FILE) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch: (\d+); kernel_source_sha256: ([0-9a-f]+)", text)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return int(m.group(1))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.rows, self.proc, self.bus_id = [], None, bus_id

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "25"]
        if self.bus_id:
            cmd[1:1] = ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:   # sampling has started before the region
                time.sleep(0.005)
            self.rows.clear()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            n = len(self.rows)
            t0 = time.time()
            while len(self.rows) <= n and time.time() - t0 < 1.0:   # one sample after the region ends
                time.sleep(0.005)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device="cpu"):
    """Largest `value` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_backend() != "nccl":
        device = "cpu"                 # gloo: host tensors
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks per second of the slowest rank (weak scaling:
    every rank runs an equal share of the job)."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores (bounded sample per step)
# ---------------------------------------------------------------------------
def oracle_sample(params, n_per_set, threads=0):
    import oracle
    from paper_2302_05170_b300 import workloads as W
    w = W.gbm_online(n_paths_per_set=n_per_set, params=params)
    t0 = time.perf_counter()
    yt = oracle.seven_league_paths(oracle.MODEL_MLP, np.asarray(w["params"], np.float64), w["theta"],
                                   w["Y0"], w["offsets"], w["T"], w["n_steps"], w["m"], w["seed"],
                                   d_in=4, threads=threads)
    dt = time.perf_counter() - t0
    path_steps = int(w["offsets"][-1]) * w["n_steps"]
    return yt, w["offsets"], path_steps, dt


def run_reference(args):
    import oracle
    from paper_2302_05170_b300 import workloads as W
    ws, rank, _ = _dist()
    if rank != 0:
        return
    oracle.build()
    params = W.xavier_params(4, 7, seed=0)
    n_per_set = args.ref_paths
    cores = oracle.num_threads()
    for _ in range(args.warmup):
        oracle_sample(params, max(n_per_set // 10, 10))
    total_ps, total_t = 0, 0.0
    for _ in range(args.steps):
        _, _, ps, dt = oracle_sample(params, n_per_set)
        total_ps += ps
        total_t += dt
    v = total_ps / total_t
    sample = "16 theta x %d paths x 16 steps per step (of 16 x 1e6)" % n_per_set
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_sets": 16,
                                            "paths_per_set": 10 ** 6, "n_steps": 16, "m": 7},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_oracle_checks(checks):
    """FP64-oracle error of each secondary result on its bounded sample (the cpu_baseline leg):
    per result the max, 99.99th percentile and mean of |a - b| / (|b| + s) over the sampled paths
    (s: the state's scale), or, for the adjoints, per component (value, d/dY0, d/dtheta) with s =
    the component's mean |b|, and the share of paths within 2e-3."""
    import oracle
    out = {}
    for c in checks:
        k = c["kind"]
        if k in ("paths", "cdcq", "cdc"):
            f = {"paths": oracle.seven_league_paths, "cdcq": oracle.cdcq_paths, "cdc": oracle.cdc_paths}[k]
            want = f(oracle.MODEL_MLP, c["P"], c["theta"], c["Y0"], c["offsets"], c["T"], c["n_steps"], c["m"],
                     c["seed"], idx=c["idx"], d_in=c["d_in"], act=c["act"])
            e = np.abs(c["got"] - want) / (np.abs(want) + c["scale"])
            out[c["name"]] = {"max": float(e.max()), "p9999": float(np.percentile(e, 99.99)), "mean": float(e.mean()),
                              "n_paths": int(len(e))}
        elif k == "labels":
            th = np.asarray(c["theta"])
            want = oracle.em_labels(2, th, c["Yi"], c["dt"], c["n_paths"], c["n_fine"], c["m"], c["seed"],
                                    n_rows=c["rows"])
            s = np.maximum(th[:c["rows"], 1], np.asarray(c["Yi"])[:c["rows"]])[:, None]
            e = np.abs(c["got"] - want) / (np.abs(want) + s)
            out[c["name"]] = {"max": float(e.max()), "mean": float(e.mean()), "n_labels": int(e.size)}
        elif k == "adjoint":
            _, val, gr = oracle.seven_league_payoff_grad(oracle.MODEL_MLP, c["P"], c["theta"], c["Y0"], c["offsets"],
                                                         c["T"], c["n_steps"], c["m"], c["seed"], c["K"],
                                                         idx=c["idx"], d_in=c["d_in"], act=c["act"])
            want = np.vstack([val[None, :], gr.T])
            res = {}
            for comp, name in enumerate(["value", "dY0"] + ["dtheta%d" % i for i in range(want.shape[0] - 2)]):
                b = want[comp]
                e = np.abs(c["got"][comp] - b) / (np.abs(b) + np.abs(b).mean() + 1e-12)
                res[name] = {"max": float(e.max()), "p999": float(np.percentile(e, 99.9)),
                             "within_2e-3": float((e <= 2e-3).mean())}
            res["n_paths"] = int(want.shape[1])
            out[c["name"]] = res
    return out


def run_labels_only(args, torch, sl, W, local):
    """Offline stage alone: em_collocation_labels on the CIR label workload."""
    sl.load()
    dev = torch.device("cuda", local)
    th, yi, dtr = W.cir_label_rows(1024)
    thd, yid, dtd = (torch.as_tensor(a, device=dev) for a in (th, yi, dtr))
    lab = torch.empty((1024, 7), dtype=torch.float32, device=dev)
    wsl = torch.empty(sl.em_labels_workspace_size(1024, 10 ** 5, 7), dtype=torch.uint8, device=dev)
    run = lambda: sl.em_collocation_labels(2, thd, yid, dtd, 10 ** 5, 100, 7, 1, labels=lab, ws=wsl)
    for _ in range(max(args.warmup, 1)):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        run()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"metric": "EM label samples/s (CIR 1024 rows x 1e5 paths x 100 fine steps, 7 quantiles)",
                      "value": 1024 * 10 ** 5 / (ms * 1e-3), "unit": "samples/s", "ms_per_step": ms,
                      "steps": args.steps, "fine_steps_per_s": 1024 * 10 ** 7 / (ms * 1e-3)}), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--paths", type=int, default=10 ** 6, help="paths per theta set")
    ap.add_argument("--ref-paths", type=int, default=2000, help="oracle paths per set per reference step")
    ap.add_argument("--cpu-paths", type=int, default=20000, help="oracle paths per set for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--weights", default="trained", choices=["trained", "xavier"])
    ap.add_argument("--only-labels", action="store_true",
                    help="time only the offline label stage (CIR, 1024 rows x 1e5 paths x 100 fine steps)")
    ap.add_argument("--train-steps", type=int, default=40000)
    ap.add_argument("--tc-config", default=None,
                    help="tensor-core launch shape 'slots/tiles-per-warpgroup' (e.g. 4/1) instead of autotuning")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2302_05170_b300 as sl
    from paper_2302_05170_b300 import sharding
    from paper_2302_05170_b300 import workloads as W

    world, rank, local = _dist()
    local = local % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(local)
    if args.only_labels:
        return run_labels_only(args, torch, sl, W, local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(os.environ.get("SL_DIST_BACKEND", "nccl"))
    sl.load()
    dev = torch.device("cuda", local)
    f32, i64 = torch.float32, torch.int64

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if args.weights == "trained":
        from paper_2302_05170_b300 import pipeline
        P_tr, losses_tr, _ = pipeline.train_gbm_online_network(n_rows=1 << 15, n_steps=args.train_steps,
                                                               **TRAIN_RECIPE)
        torch.cuda.synchronize()
        params_np = P_tr.cpu().numpy()
        weights_kind = ("trained on the GPU: em_collocation_labels (GBM, 32768 rows x 4e5 paths x 100 fine "
                        "steps, dt in {0.125,0.25,0.5,1}), %d Adam steps on normalised features and labels "
                        "(folded into the first and last layers), then 10000 Adam steps of the BF16-rounded "
                        "network; every weight is a BF16 value and both forms run it" % args.train_steps)
    else:
        params_np = W.xavier_params(4, 7, seed=0)
        weights_kind = "Xavier-uniform seed 0 (untrained)"
    # the job: 16 parameter sets per rank; rank r runs its contiguous share of the flat path list
    n_sets_job = 16 * world
    w = W.gbm_online(n_paths_per_set=args.paths, n_sets=n_sets_job, params=params_np)
    seed = w["seed"]
    total_job = int(w["offsets"][-1])
    first, total = sharding.rank_range(total_job, world, rank)
    n_steps, m, T = w["n_steps"], w["m"], w["T"]
    theta = torch.as_tensor(w["theta"], device=dev)
    Y0 = torch.as_tensor(w["Y0"], device=dev)
    off = torch.as_tensor(w["offsets"], device=dev)
    P = torch.as_tensor(w["params"], device=dev)
    prec = sl.PREC_BF16 if args.prec == "bf16" else sl.PREC_FP32
    net = sl.make_net(P, 4, 7, prec=prec)
    yt = torch.empty(total, dtype=f32, device=dev)
    mean = torch.empty(n_sets_job, dtype=torch.float64, device=dev)
    var = torch.empty_like(mean)
    ws = torch.empty(max(sl.simulate_workspace_size(total, n_sets_job),
                         sl.simulate_range_workspace_size(total, n_sets_job)), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    stream = torch.cuda.current_stream()

    def step(out_yt=yt, out_mean=mean, out_var=var, net_=net):
        if world == 1:
            sl.seven_league_simulate_batched(sl.MODEL_MLP, net_, theta, Y0, off, T, n_steps, m, seed,
                                             out_YT=out_yt, out_mean=out_mean, out_var=out_var, ws=ws,
                                             total_paths=total)
            return None
        # this rank's range, then one all-gather of the per-set partial moments (NCCL)
        r = sharding.simulate_sharded(sl.MODEL_MLP, net_, theta, Y0, off, T, n_steps, m, seed,
                                      total_paths=total_job, out_YT=out_yt, ws=ws)
        if out_mean is not None:
            out_mean.copy_(torch.as_tensor(r["mean"]), non_blocking=True)
        if out_var is not None:
            out_var.copy_(torch.as_tensor(r["var"]), non_blocking=True)
        return r

    tuning = None
    if prec == sl.PREC_BF16 and args.tc_config:   # a fixed launch shape (profiling), no autotuning
        slots, tpw = (int(x) for x in args.tc_config.split("/"))
        sl.tc_set_pipeline(1)
        sl.tc_set_slots(slots)
        sl.tc_set_pipeline(tpw)
        tuning = {"tc_slots": slots, "tc_tiles_per_warpgroup": tpw, "ms_by_config": None}
    elif prec == sl.PREC_BF16:
        from paper_2302_05170_b300 import autotune
        best, tms = autotune.tune_slots(lambda: step(out_mean=None, out_var=None),
                                        "gbm-online d4 m7 s16 n%d" % total, use_cache=False)
        tuning = {"tc_slots": best[0], "tc_tiles_per_warpgroup": best[1], "ms_by_config": tms}
    for _ in range(max(args.warmup, 3)):
        step()
    assert sl.workspace_status(ws) == 0, "device status set during warm-up"
    # --- timed region: K steps, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except Exception:
        pass
    barrier()
    with ClockSampler(bus) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(ms) / 1e3
    t_max = max_over_ranks(t_local, dev)
    path_steps = total * n_steps
    value = whole_job_rate(path_steps * args.steps, world, t_max)
    # 7L kernel + 2 moment kernels (a rank of a split job: + the range-offsets kernel)
    launches_per_step = 3 if world == 1 else 4

    def kernel_only():
        if world == 1:
            step(out_mean=None, out_var=None)
        else:
            sl.seven_league_simulate_range(sl.MODEL_MLP, net, theta, Y0, off, T, n_steps, m, seed, first, total,
                                           out_YT=yt, ws=ws)

    # --- dominant kernel alone (Y_T only: status clear + the 7L kernel)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in kev:
        flush.zero_()
        a.record(stream)
        kernel_only()
        b.record(stream)
    torch.cuda.synchronize()
    k_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
    peaks, peak_src = _peaks()
    if prec == sl.PREC_BF16:
        achieved = ALG_FLOPS_PER_PATH_STEP * path_steps / (k_ms * 1e-3) / 1e12
        # the kernel is timed alone in launches of ~10 ms at the maximum clock (the clock record
        # below shows no power-cap reason): the burst figure is its peak; the power-capped
        # sustained figure is reported beside it as a note only
        peak = peaks["bf16_tflops"]
        default_workload = (args.paths, n_steps, m) == (10 ** 6, 16, 7)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": recorded_traffic() if default_workload else None,
                "peak_kind": "bf16 burst, " + peak_src,
                "note_frac_of_sustained": achieved / peaks["bf16_tflops_sustained"]}
    else:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        achieved = ALG_FLOPS_PER_PATH_STEP * path_steps / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_kind": "FP32 FMA: %d SMs x 128 lanes x 2 flop x %.0f MHz" % (sms, peaks["sm_max_mhz"])}

    secondary = {}
    checks = []          # FP64-oracle checks of the secondary results, run in the cpu_baseline leg
    if not args.no_secondary and rank == 0 and world == 1:
        # the other form on the same paths
        other = sl.PREC_FP32 if prec == sl.PREC_BF16 else sl.PREC_BF16
        try:
            net_o = sl.make_net(P, 4, 7, prec=other)
            yt_o = torch.empty_like(yt)
            step(out_yt=yt_o, net_=net_o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                step(out_yt=yt_o, net_=net_o)
            e1.record(stream)
            torch.cuda.synchronize()
            o_ms = e0.elapsed_time(e1) / 3
            key = "fp32_simt" if other == sl.PREC_FP32 else "bf16_tc"
            secondary[key + "_path_steps_per_s"] = path_steps / (o_ms * 1e-3)
            if other == sl.PREC_FP32:   # the FP32 form against its own roofline (FP32 FMA lanes)
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                fp32_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
                secondary["fp32_simt_roofline_frac"] = (ALG_FLOPS_PER_PATH_STEP * path_steps / (o_ms * 1e-3) / 1e12
                                                        / fp32_peak)
            secondary["bf16_over_fp32"] = (value / (path_steps / (o_ms * 1e-3))) if other == sl.PREC_FP32 else \
                (path_steps / (o_ms * 1e-3)) / value
            a64, b64 = yt.double(), yt_o.double()
            dd = (a64 - b64).abs() / (b64.abs() + 1.0)
            secondary["bf16_vs_fp32_max_rel_diff"] = float(dd.max())
            secondary["bf16_vs_fp32_p9999_rel_diff"] = float(torch.quantile(dd[::16], 0.9999))
            secondary["bf16_vs_fp32_weights"] = "the same BF16-valued weights in both forms" if \
                args.weights == "trained" else "the same FP32 weights (BF16-rounded in the tensor-core form)"
            # both forms against the exact-collocation GBM chain on the same normals (the network's error)
            yt_x = torch.empty_like(yt)
            sl.seven_league_simulate_batched(sl.MODEL_GBM_EXACT, None, theta, Y0, off, T, n_steps, m, seed,
                                             out_YT=yt_x, total_paths=total)
            x64 = yt_x.double()
            for key_f, y64 in (("bf16", a64 if prec == sl.PREC_BF16 else b64), ("fp32", b64 if prec == sl.PREC_BF16 else a64)):
                e = (y64 - x64).abs()
                secondary["err_vs_exact_map_" + key_f] = {"mean_abs": float(e.mean()),
                                                           "p9999_abs": float(torch.quantile(e[::16], 0.9999)),
                                                           "max_abs": float(e.max())}
            secondary["err_vs_exact_map_note"] = ("|Y_T - Y_T(exact GBM collocation map)| per path, same normals, "
                                                  "all 16e6 paths (p99.99 on every 16th): the trained network's own "
                                                  "error, the same in both forms")
            del yt_x
            fp32_yt = (yt_o if other == sl.PREC_FP32 else yt)
            ix = sample_idx(w["offsets"], 200)
            checks.append(dict(name="fp32_form", kind="paths", P=params_np, theta=w["theta"], Y0=w["Y0"],
                               offsets=w["offsets"], T=T, n_steps=n_steps, m=m, seed=seed, d_in=4, act=0,
                               idx=ix, got=take(fp32_yt, ix), scale=1.0))
        except sl.SLError as e:
            secondary["other_form_error"] = str(e)
        if prec == sl.PREC_BF16:
            # the same workload with the paper's Softplus activation in the tensor-core form
            # (log(1 + e^z) on the fast exponent/logarithm unit in the epilogue)
            if args.weights == "trained":
                P_sp, _, _ = pipeline.train_gbm_online_network(n_rows=1 << 15, n_steps=args.train_steps, act=1,
                                                               dts=ADJ_DTS, **TRAIN_RECIPE)
            else:
                P_sp = P
            net_sp = sl.make_net(P_sp, 4, 7, act=sl.ACT_SOFTPLUS, prec=sl.PREC_BF16)
            yt_sp = torch.empty_like(yt)
            step(out_yt=yt_sp, net_=net_sp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                step(out_yt=yt_sp, net_=net_sp)
            e1.record(stream)
            torch.cuda.synchronize()
            secondary["softplus_bf16_path_steps_per_s"] = path_steps / (e0.elapsed_time(e1) / 3 * 1e-3)
            ix = sample_idx(w["offsets"], 200)
            checks.append(dict(name="softplus_bf16", kind="paths", P=W.bf16_round(P_sp.cpu().numpy()), theta=w["theta"],
                               Y0=w["Y0"], offsets=w["offsets"], T=T, n_steps=n_steps, m=m, seed=seed, d_in=4,
                               act=1, idx=ix, got=take(yt_sp, ix), scale=1.0))
            del yt_sp
        # the 7L-CDC variant on the same paths (Table 6.1's second scheme): the network only at the
        # marginal collocation points of each (set, step), an interpolation in Y per path.  With a
        # network (trained weights: the GBM network trained again over the horizons 0.125 .. 2, so
        # that it gives the marginal points too; otherwise workloads.near_affine_params, outputs
        # shaped like collocation points -- an untrained Xavier network's marginal points are
        # unordered) and with the exact GBM map.
        if args.weights == "trained":
            P_cdc, _, _ = pipeline.train_gbm_online_network(n_rows=1 << 15, n_steps=args.train_steps,
                                                            dts=tuple(0.125 * np.arange(1, 17)), **TRAIN_RECIPE)
            cdc_net_kind = ("GBM network trained over the horizons 0.125..2 (%d Adam steps, the bench's training "
                            "recipe)" % args.train_steps)
        else:
            P_cdc = torch.as_tensor(W.near_affine_params(4, 7, seed=0), device=dev)
            cdc_net_kind = "workloads.near_affine_params (seed 0)"
        net_cdc = sl.make_net(P_cdc, 4, 7)
        ws_cdc = torch.empty(sl.cdc_workspace_size(total, 16, n_steps), dtype=torch.uint8, device=dev)
        yt_c = torch.empty_like(yt)
        mean_c = torch.empty_like(mean)
        for model_c, space_c, key in ((sl.MODEL_MLP, sl.CDC_QUANTILE, "cdc"), (sl.MODEL_GBM_EXACT, sl.CDC_QUANTILE,
                                                                              "cdc_gbm_exact"),
                                      (sl.MODEL_MLP, sl.CDC_Y, "cdc_y")):
            net_c = net_cdc if model_c == sl.MODEL_MLP else None
            run_c = lambda: sl.seven_league_cdc_simulate_batched(model_c, net_c, theta, Y0, off, T, n_steps, m, seed,
                                                                 space=space_c, out_YT=yt_c, out_mean=mean_c,
                                                                 ws=ws_cdc, total_paths=total)
            run_c()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                run_c()
            e1.record(stream)
            torch.cuda.synchronize()
            if sl.workspace_status(ws_cdc) != 0:
                secondary[key + "_error"] = "device status %d" % sl.workspace_status(ws_cdc)
                continue
            c_rate = path_steps / (e0.elapsed_time(e1) / 5 * 1e-3)
            secondary[key + "_path_steps_per_s"] = c_rate
            if model_c == sl.MODEL_MLP:
                ix = sample_idx(w["offsets"], 125)
                checks.append(dict(name=key, kind="cdcq" if space_c == sl.CDC_QUANTILE else "cdc",
                                   P=P_cdc.cpu().numpy(), theta=w["theta"], Y0=w["Y0"], offsets=w["offsets"], T=T,
                                   n_steps=n_steps, m=m, seed=seed, d_in=4, act=0, idx=ix, got=take(yt_c, ix),
                                   scale=1.0))
            if key == "cdc":
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                fp32_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6
                secondary["cdc_fp32_roofline_frac"] = CDC_FLOPS_PER_PATH_STEP * c_rate / fp32_peak
                secondary["cdc_over_7l_bf16"] = c_rate / value
        secondary["cdc_workload"] = ("7L-CDC on the GBM workload above (16 sets x %d paths x %d steps, m=7); tables "
                                     "of network evaluations per (set, step), then 2 paths per thread; cdc: in the "
                                     "marginal's quantile coordinate, cdc_y: interpolation in Y; network: %s"
                                     % (args.paths, n_steps, cdc_net_kind))
        if args.weights == "trained" and "cdc_error" not in secondary:
            # accuracy on every path against the exact-collocation GBM chain on the same normals:
            # the 7L-CDC scheme and the 7L scheme (BF16 form) with the same network
            yt_ex = torch.empty_like(yt)
            sl.seven_league_simulate_batched(sl.MODEL_GBM_EXACT, None, theta, Y0, off, T, n_steps, m, seed,
                                             out_YT=yt_ex, total_paths=total)
            ex = yt_ex.double()
            for space_c, key in ((sl.CDC_QUANTILE, "cdc"), (sl.CDC_Y, "cdc_y")):
                sl.seven_league_cdc_simulate_batched(sl.MODEL_MLP, net_cdc, theta, Y0, off, T, n_steps, m, seed,
                                                     space=space_c, out_YT=yt_c, ws=ws_cdc, total_paths=total)
                secondary[key + "_mean_abs_err_vs_exact_map"] = float((yt_c.double() - ex).abs().mean().item())
            yt_7 = torch.empty_like(yt)
            sl.seven_league_simulate_batched(sl.MODEL_MLP, sl.make_net(P_cdc, 4, 7, prec=sl.PREC_BF16), theta, Y0,
                                             off, T, n_steps, m, seed, out_YT=yt_7, total_paths=total)
            secondary["7l_same_network_mean_abs_err_vs_exact_map"] = float((yt_7.double() - ex).abs().mean().item())
            del yt_ex, yt_7
        del yt_c, ws_cdc
        # offline stage: EM label samples/s on the CIR labels workload
        th, yi, dtr = W.cir_label_rows(1024)
        thd, yid, dtd = (torch.as_tensor(a, device=dev) for a in (th, yi, dtr))
        lab = torch.empty((1024, 7), dtype=f32, device=dev)
        wsl = torch.empty(sl.em_labels_workspace_size(1024, 10 ** 5, 7), dtype=torch.uint8, device=dev)
        sl.em_collocation_labels(2, thd, yid, dtd, 10 ** 5, 100, 7, 1, labels=lab, ws=wsl)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            sl.em_collocation_labels(2, thd, yid, dtd, 10 ** 5, 100, 7, 1, labels=lab, ws=wsl)
        e1.record(stream)
        torch.cuda.synchronize()
        l_ms = e0.elapsed_time(e1) / 3
        secondary["em_label_samples_per_s"] = 1024 * 10 ** 5 / (l_ms * 1e-3)
        secondary["em_fine_steps_per_s"] = 1024 * 10 ** 5 * 100 / (l_ms * 1e-3)
        secondary["em_labels_workload"] = "CIR 1024 rows x 1e5 paths x 100 fine steps, 7 quantiles"
        checks.append(dict(name="em_labels", kind="labels", theta=th, Yi=yi, dt=dtr, n_paths=10 ** 5, n_fine=100,
                           m=7, seed=1, rows=4, got=lab[:4].double().cpu().numpy()))
        del wsl
        # CIR network trained on those labels, then the batched CIR workload: 4096 theta sets with
        # log-uniform path counts in [1e3, 1e5], 32 steps, in one persistent launch replayed from a
        # captured CUDA graph
        from paper_2302_05170_b300 import pipeline
        feats_c = torch.cat([yid[:, None], dtd[:, None], thd], 1).contiguous()
        P_c = torch.as_tensor(W.xavier_params(5, 7, seed=0), device=dev)
        am_c, av_c = torch.zeros_like(P_c), torch.zeros_like(P_c)
        rows_all = [torch.as_tensor(W.minibatch_rows(1024, 1024, 1000, seed=40 + c), device=dev) for c in range(10)]
        t_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        t_ev[0].record(stream)
        for c in range(10):
            sl.train(P_c, 5, 7, am_c, av_c, 1000 * c, feats_c, lab, rows_all[c], 1024, lr=1e-3 * 0.01 ** (c / 9))
        t_ev[1].record(stream)
        torch.cuda.synchronize()
        secondary["train_adam_steps_per_s"] = 10000 / (t_ev[0].elapsed_time(t_ev[1]) * 1e-3)
        secondary["train_workload"] = ("CIR network 5->50x4->7, batch 1024 of 1024 label rows, 10000 Adam steps "
                                       "(forward, MSE back-propagation, deterministic reduction, update)")
        cb = W.cir_batched()
        tot_c = int(cb["offsets"][-1])
        net_c = sl.make_net(P_c, 5, 7, prec=prec)
        th_c, y0_c = torch.as_tensor(cb["theta"], device=dev), torch.as_tensor(cb["Y0"], device=dev)
        off_c = torch.as_tensor(cb["offsets"], device=dev)
        yt_c = torch.empty(tot_c, dtype=f32, device=dev)
        mean_c = torch.empty(4096, dtype=torch.float64, device=dev)
        var_c = torch.empty_like(mean_c)
        ws_c = torch.empty(sl.simulate_workspace_size(tot_c, 4096), dtype=torch.uint8, device=dev)
        run_c = lambda: sl.seven_league_simulate_batched(sl.MODEL_MLP, net_c, th_c, y0_c, off_c, cb["T"],
                                                         cb["n_steps"], 7, cb["seed"], out_YT=yt_c,
                                                         out_mean=mean_c, out_var=var_c, ws=ws_c,
                                                         total_paths=tot_c)
        run_c()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run_c()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        c_ms = e0.elapsed_time(e1) / 3
        assert sl.workspace_status(ws_c) == 0
        secondary["cir_batched_path_steps_per_s"] = tot_c * cb["n_steps"] / (c_ms * 1e-3)
        ix = sample_idx(cb["offsets"], 2)
        P_c_np = P_c.cpu().numpy()
        checks.append(dict(name="cir_batched", kind="paths", P=W.bf16_round(P_c_np) if prec == sl.PREC_BF16 else P_c_np,
                           theta=cb["theta"], Y0=cb["Y0"], offsets=cb["offsets"], T=cb["T"], n_steps=cb["n_steps"],
                           m=7, seed=cb["seed"], d_in=5, act=0, idx=ix, got=take(yt_c, ix), scale=0.1))
        secondary["cir_batched_workload"] = ("CIR 4096 theta sets, %d paths (log-uniform 1e3..1e5 per set), "
                                             "32 steps, m=7, one persistent launch in a CUDA graph" % tot_c)
        del ws_c
        # the same batch through the 7L-CDC scheme (quantile coordinate; 4096 x 32 table entries):
        # timing only, with workloads.near_affine_params (the CIR network is trained for steps of
        # 0.1..1, not for the horizons up to T = 8 the marginal points need)
        P_cc = torch.as_tensor(W.near_affine_params(5, 7, seed=0), device=dev)
        net_cc = sl.make_net(P_cc, 5, 7)
        ws_cc = torch.empty(sl.cdc_workspace_size(tot_c, 4096, cb["n_steps"]), dtype=torch.uint8, device=dev)
        run_cc = lambda: sl.seven_league_cdc_simulate_batched(sl.MODEL_MLP, net_cc, th_c, y0_c, off_c, cb["T"],
                                                              cb["n_steps"], 7, cb["seed"], out_YT=yt_c,
                                                              out_mean=mean_c, ws=ws_cc, total_paths=tot_c)
        run_cc()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            run_cc()
        e1.record(stream)
        torch.cuda.synchronize()
        if sl.workspace_status(ws_cc) == 0:
            secondary["cdc_cir_batched_path_steps_per_s"] = tot_c * cb["n_steps"] / (e0.elapsed_time(e1) / 3 * 1e-3)
            ix = sample_idx(cb["offsets"], 1)
            checks.append(dict(name="cdc_cir_batched", kind="cdcq", P=P_cc.cpu().numpy(), theta=cb["theta"],
                               Y0=cb["Y0"], offsets=cb["offsets"], T=cb["T"], n_steps=cb["n_steps"], m=7,
                               seed=cb["seed"], d_in=5, act=0, idx=ix, got=take(yt_c, ix), scale=0.1))
        else:
            secondary["cdc_cir_batched_error"] = "device status %d" % sl.workspace_status(ws_cc)
        del yt_c, ws_cc
        # adjoint: GBM mu = 0.1, sigma = 0.3, Y0 = 1, T = 1 in 64 steps (dt = 1/64), 1e6 paths, checkpoint
        # every 8 steps, call K = 1.  The networks are trained down to dt = 1/64 (ReLU, FP32 and BF16
        # forms; the Softplus network trained as such, BF16 form); the exact GBM collocation map on the
        # same normals gives the scheme's value without a network's error; Black-Scholes (undiscounted)
        # is the limit of both.  Each value is the FP64 mean over the paths, with its standard error.
        if args.weights == "trained":
            P_adj, _, _ = pipeline.train_gbm_online_network(n_rows=1 << 15, n_steps=args.train_steps, dts=ADJ_DTS,
                                                            **TRAIN_RECIPE)
        else:
            P_adj = P
        n_a, T_a, K_a, mu_a, sg_a = 10 ** 6, 1.0, 1.0, 0.1, 0.3
        off_a = torch.as_tensor(W.offsets_from_counts([n_a]), device=dev)
        th_a = torch.tensor([[mu_a, sg_a]], device=dev)
        y0_a = torch.ones(1, device=dev)
        ws_a = torch.empty(sl.adjoint_workspace_size(n_a, 1, 64, 8, 2), dtype=torch.uint8, device=dev)
        paths_a = torch.empty((4, n_a), dtype=f32, device=dev)
        per_path_a = {}
        ncdf = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
        d1 = (math.log(1.0 / K_a) + (mu_a + 0.5 * sg_a ** 2) * T_a) / (sg_a * math.sqrt(T_a))
        secondary["adjoint_black_scholes"] = {
            "value": math.exp(mu_a * T_a) * ncdf(d1) - K_a * ncdf(d1 - sg_a * math.sqrt(T_a)),
            "dY0": math.exp(mu_a * T_a) * ncdf(d1), "dmu": T_a * math.exp(mu_a * T_a) * ncdf(d1),
            "dsigma": math.exp(mu_a * T_a) * math.exp(-0.5 * d1 * d1) / math.sqrt(2 * math.pi) * math.sqrt(T_a)}
        for key, model_a, Pa, act_a, pr in (
                ("adjoint_fp32", sl.MODEL_MLP, P_adj, sl.ACT_RELU, sl.PREC_FP32),
                ("adjoint_bf16", sl.MODEL_MLP, P_adj, sl.ACT_RELU, sl.PREC_BF16),
                ("adjoint_bf16_softplus", sl.MODEL_MLP, P_sp, sl.ACT_SOFTPLUS, sl.PREC_BF16),
                ("adjoint_exact_map", sl.MODEL_GBM_EXACT, None, 0, sl.PREC_FP32)):
            net_a = sl.make_net(Pa, 4, 7, act=act_a, prec=pr) if model_a == sl.MODEL_MLP else None
            run_a = lambda: sl.seven_league_adjoint(model_a, net_a, th_a, y0_a, off_a, T_a, 64, 7, 1, K_a, ckpt_k=8,
                                                    out_paths=paths_a, ws=ws_a, total_paths=n_a)
            run_a()
            torch.cuda.synchronize()
            e0.record(stream)
            v_a, d0_a, dth_a = run_a()
            e1.record(stream)
            torch.cuda.synchronize()
            assert sl.workspace_status(ws_a) == 0
            secondary[key + "_path_steps_per_s"] = n_a * 64 / (e0.elapsed_time(e1) * 1e-3)
            se = (paths_a.double().std(dim=1) / math.sqrt(n_a)).tolist()
            vals = [v_a.item(), d0_a.item()] + dth_a[0].tolist()
            secondary[key + "_result"] = {k: [round(a, 6), round(b, 6)] for k, a, b in
                                          zip(("value", "dY0", "dmu", "dsigma"), vals, se)}
            per_path_a[key] = paths_a.double().clone()
            if model_a == sl.MODEL_MLP:
                ix = sample_idx(W.offsets_from_counts([n_a]), 2000)
                Pn = Pa.cpu().numpy()
                checks.append(dict(name=key, kind="adjoint", P=W.bf16_round(Pn) if pr == sl.PREC_BF16 else Pn,
                                   theta=[[mu_a, sg_a]], Y0=[1.0], offsets=W.offsets_from_counts([n_a]), T=T_a,
                                   n_steps=64, m=7, seed=1, K=K_a, d_in=4, act=act_a, idx=ix,
                                   got=paths_a[:, torch.as_tensor(ix, device=dev)].double().cpu().numpy()))
        secondary["adjoint_workload"] = ("GBM mu=0.1 sigma=0.3 Y0=1, 1e6 paths x 64 steps of dt=1/64, checkpoint "
                                         "every 8, call K=1; each *_result is [FP64 mean, standard error] of the "
                                         "value and its derivatives in Y0, mu, sigma; networks trained over dt "
                                         "1/64..1 (adjoint_bf16_softplus: a Softplus network trained as such); "
                                         "adjoint_exact_map: the exact GBM collocation map on the same normals")
        # each network's own error, stated per result: per path, the network chain's payoff and its
        # derivatives minus the exact map's on the same normals (paired, so the Monte Carlo noise
        # they share cancels); [mean, standard error].  A network result = the exact map's (itself
        # within its standard error of Black-Scholes) + this error.
        ex_a = per_path_a.pop("adjoint_exact_map")
        for key, pp in per_path_a.items():
            dd = pp - ex_a
            secondary[key + "_network_error"] = {
                k: [round(a, 6), round(b, 6)] for k, a, b in
                zip(("value", "dY0", "dmu", "dsigma"), dd.mean(dim=1).tolist(),
                    (dd.std(dim=1) / math.sqrt(n_a)).tolist())}
        del paths_a, per_path_a, ex_a
        # CIR adjoint on the trained CIR network (BF16 tcgen05 form): kappa=1, ybar=0.1, gamma=0.3,
        # Y0=0.1, 1e6 paths x 64 steps of dt=0.25 (inside the label rows' dt range), checkpoint every 8;
        # call K=1 lies far above the CIR range (every sensitivity is 0), K=ybar is the meaningful case
        th_ca = torch.tensor([[1.0, 0.1, 0.3]], device=dev)
        y0_ca = torch.tensor([0.1], device=dev)
        ws_ca = torch.empty(sl.adjoint_workspace_size(n_a, 1, 64, 8, 3), dtype=torch.uint8, device=dev)
        paths_ca = torch.empty((5, n_a), dtype=f32, device=dev)
        for Kc, key in ((1.0, "cir_adjoint_K1"), (0.1, "cir_adjoint_Kybar")):
            run_ca = lambda: sl.seven_league_adjoint(sl.MODEL_MLP, net_c, th_ca, y0_ca, off_a, 16.0, 64, 7, 1, Kc,
                                                     ckpt_k=8, out_paths=paths_ca, ws=ws_ca, total_paths=n_a)
            run_ca()
            torch.cuda.synchronize()
            e0.record(stream)
            v_c, d0_c, dth_c = run_ca()
            e1.record(stream)
            torch.cuda.synchronize()
            assert sl.workspace_status(ws_ca) == 0
            secondary[key + "_path_steps_per_s"] = n_a * 64 / (e0.elapsed_time(e1) * 1e-3)
            secondary[key + "_result"] = ("value %.6f dY0 %.5f dtheta %s"
                                          % (v_c.item(), d0_c.item(), [round(x, 5) for x in dth_c[0].tolist()]))
            if Kc < 1.0:
                ix = sample_idx(W.offsets_from_counts([n_a]), 2000)
                Pn = P_c.cpu().numpy()
                checks.append(dict(name=key, kind="adjoint", P=W.bf16_round(Pn) if prec == sl.PREC_BF16 else Pn,
                                   theta=[[1.0, 0.1, 0.3]], Y0=[0.1], offsets=W.offsets_from_counts([n_a]), T=16.0,
                                   n_steps=64, m=7, seed=1, K=Kc, d_in=5, act=0, idx=ix,
                                   got=paths_ca[:, torch.as_tensor(ix, device=dev)].double().cpu().numpy()))
        secondary["cir_adjoint_workload"] = ("CIR network (BF16 tcgen05), kappa=1 ybar=0.1 gamma=0.3 Y0=0.1, "
                                             "1e6 paths x 64 steps of dt=0.25, checkpoint every 8")
        # the paper's own experiment (Table 6.1's path counts): OU, m = 5, trained network (over the
        # horizons 0.125 .. 2, so that it also gives the 7L-CDC scheme its marginal points); time per
        # run of 16 steps (T = 2) for the 7L scheme in both forms and for the 7L-CDC scheme, and the
        # pathwise error at 2e5 paths against Eq. (6.6) on the same normals (exact OU model)
        P_ou, _, _ = pipeline.train_ou_network(n_rows=1 << 14, n_steps=20000, dts=tuple(0.125 * np.arange(1, 17)),
                                               device=dev)
        th_ou, y0_ou = torch.tensor([[0.5, 0.3, 1.0]], device=dev), torch.tensor([1.5], device=dev)
        ou_ms, ou_graph_ms = {}, {}
        for pr, key in ((sl.PREC_BF16, "bf16"), (sl.PREC_FP32, "fp32"), (sl.PREC_FP32, "cdc"), (sl.PREC_FP32, "cdc_y")):
            net_ou = sl.make_net(P_ou, 5, 5, prec=pr)
            for n_ou in (1000, 50000, 100000, 200000):
                off_ou = torch.as_tensor(W.offsets_from_counts([n_ou]), device=dev)
                yt_ou = torch.empty(n_ou, dtype=f32, device=dev)
                if key.startswith("cdc"):
                    ws_ou = torch.empty(sl.cdc_workspace_size(n_ou, 1, 16), dtype=torch.uint8, device=dev)
                    sp_ou = sl.CDC_Y if key == "cdc_y" else sl.CDC_QUANTILE
                    run_ou = lambda: sl.seven_league_cdc_simulate_batched(sl.MODEL_MLP, net_ou, th_ou, y0_ou, off_ou,
                                                                          2.0, 16, 5, 3, space=sp_ou, out_YT=yt_ou,
                                                                          ws=ws_ou, total_paths=n_ou)
                else:
                    ws_ou = torch.empty(sl.simulate_workspace_size(n_ou, 1), dtype=torch.uint8, device=dev)
                    run_ou = lambda: sl.seven_league_simulate_batched(sl.MODEL_MLP, net_ou, th_ou, y0_ou, off_ou, 2.0,
                                                                      16, 5, 3, out_YT=yt_ou, ws=ws_ou,
                                                                      total_paths=n_ou)
                run_ou()
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(10):
                    run_ou()
                e1.record(stream)
                torch.cuda.synchronize()
                ou_ms["%s_%d" % (key, n_ou)] = round(e0.elapsed_time(e1) / 10, 4)
                # the same run replayed from a CUDA graph: device time without the Python binding's
                # per-call host work
                try:
                    g_ou = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g_ou):
                        run_ou()
                    g_ou.replay()
                    torch.cuda.synchronize()
                    e0.record(stream)
                    for _ in range(10):
                        g_ou.replay()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ou_graph_ms["%s_%d" % (key, n_ou)] = round(e0.elapsed_time(e1) / 10, 4)
                    del g_ou
                except RuntimeError as e:
                    ou_graph_ms["%s_%d" % (key, n_ou)] = "not captured: %s" % str(e)[:80]
            ix = sample_idx(W.offsets_from_counts([n_ou]), 3000)
            Pn = P_ou.cpu().numpy()
            checks.append(dict(name="ou_" + key, kind="cdcq" if key == "cdc" else ("cdc" if key == "cdc_y" else "paths"),
                               P=W.bf16_round(Pn) if pr == sl.PREC_BF16 and key == "bf16" else Pn,
                               theta=[[0.5, 0.3, 1.0]], Y0=[1.5], offsets=W.offsets_from_counts([n_ou]), T=2.0,
                               n_steps=16, m=5, seed=3, d_in=5, act=0, idx=ix, got=take(yt_ou, ix), scale=1.5))
            yt_ex = torch.empty(200000, dtype=f32, device=dev)
            sl.seven_league_simulate_batched(sl.MODEL_OU_EXACT, None, th_ou, y0_ou, off_ou, 2.0, 16, 5, 3,
                                             out_YT=yt_ex, total_paths=200000)
            secondary["ou_pathwise_err_" + key] = float((yt_ou - yt_ex).abs().mean().item())
        secondary["ou_table61_ms_per_run"] = ou_ms
        secondary["ou_table61_graph_ms_per_run"] = ou_graph_ms
        secondary["ou_table61_workload"] = ("OU (Ybar 0.5, sigma 0.3, lambda 1, Y0 1.5), m=5, trained 5->50x4->5 ReLU "
                                            "network (horizons 0.125..2), T=2 in 16 steps; paths 1e3/5e4/1e5/2e5 as "
                                            "in Table 6.1; keys bf16/fp32 = 7L scheme, cdc / cdc_y = 7L-CDC scheme (quantile coordinate / Y); "
                                            "ms_per_run: ten calls through the Python binding, graph_ms_per_run: "
                                            "ten replays of a CUDA graph of one call")

    # --- end to end through the C ABI with host buffers (pinned), copies timed.  Every step copies
    # its inputs host -> device, runs the sampler and copies Y_T and the set moments back; the steps
    # are pipelined as a user streaming results would: the result copy of step k runs on a copy
    # stream while step k+1 samples into the other of two device buffers.
    h_theta = torch.as_tensor(w["theta"]).pin_memory()
    h_y0 = torch.as_tensor(w["Y0"]).pin_memory()
    h_off = torch.as_tensor(w["offsets"]).pin_memory()
    h_P = torch.as_tensor(w["params"]).pin_memory()
    yt_b = [yt, torch.empty_like(yt)]
    h_yt_b = [torch.empty(total, dtype=f32).pin_memory() for _ in range(2)]
    mom_b = [torch.empty(2 * n_sets_job, dtype=torch.float64, device=dev) for _ in range(2)]
    h_mom_b = [torch.empty(2 * n_sets_job, dtype=torch.float64).pin_memory() for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in (h_theta, h_y0, h_off, h_P))
    d2h = h_yt_b[0].numel() * 4 + h_mom_b[0].numel() * 8
    copy_stream = torch.cuda.Stream(device=dev)

    def e2e_steps(n):
        done = [None, None]
        for k in range(n):
            j = k % 2
            if done[j] is not None:
                stream.wait_event(done[j])          # buffer j's previous result has left the device
            theta.copy_(h_theta, non_blocking=True)
            Y0.copy_(h_y0, non_blocking=True)
            off.copy_(h_off, non_blocking=True)
            P.copy_(h_P, non_blocking=True)
            step(out_yt=yt_b[j], out_mean=mom_b[j][:n_sets_job], out_var=mom_b[j][n_sets_job:])
            ready = torch.cuda.Event()
            ready.record(stream)
            copy_stream.wait_event(ready)
            with torch.cuda.stream(copy_stream):
                h_yt_b[j].copy_(yt_b[j], non_blocking=True)
                h_mom_b[j].copy_(mom_b[j], non_blocking=True)
            done[j] = torch.cuda.Event()
            done[j].record(copy_stream)
        for d in done:
            if d is not None:
                stream.wait_event(d)

    e2e_steps(2)                                    # warm-up
    torch.cuda.synchronize()
    n_e2e = max(3, args.steps)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    e2e_steps(n_e2e)
    b.record(stream)
    b.synchronize()
    e2e_ms = [a.elapsed_time(b) / n_e2e]
    assert np.array_equal(h_yt_b[(n_e2e - 1) % 2].numpy(), yt_b[(n_e2e - 1) % 2].cpu().numpy())
    e2e_value = whole_job_rate(path_steps, world, max_over_ranks(float(np.mean(e2e_ms)) * 1e-3, dev))

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        n_s = min(args.cpu_paths, args.paths)
        # the oracle runs with the weights the form uses (BF16-valued for the tensor-core form)
        Pw = W.bf16_round(params_np) if prec == sl.PREC_BF16 else params_np
        yo, offs_o, ps, dt = oracle_sample(Pw, n_s)
        cpu = {"value": ps / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "first %d paths of each of the 16 theta sets, 16 steps (%d path-steps, %.1f s)"
                         % (n_s, ps, dt)}
        # accuracy of this run's Y_T on the sampled paths (same seed and weights)
        idx = np.concatenate([np.arange(s * args.paths, s * args.paths + n_s) for s in range(16)])
        g = yt.cpu().numpy()[idx].astype(np.float64)
        err = np.abs(g - yo) / (np.abs(yo) + 1.0)
        accuracy = {"max_rel_err": float(err.max()), "p9999_rel_err": float(np.percentile(err, 99.99)),
                    "n_paths_checked": int(len(idx)), "metric": "|a-b|/(|b|+Y0) vs FP64 oracle"}
        if checks:
            t_chk = time.perf_counter()
            secondary["oracle_err"] = run_oracle_checks(checks)
            secondary["oracle_err_note"] = ("every secondary result against the FP64 oracle on a bounded sample of "
                                            "its paths (same weights, normals and inputs): max / p99.99 / mean of "
                                            "|a-b|/(|b|+s); adjoints per component with s = mean |b| (%.1f s)"
                                            % (time.perf_counter() - t_chk))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if prec == sl.PREC_BF16 else "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if world == 1 else
                           "%s; one job of %d theta sets split across %d ranks by path count, per-set "
                           "moments combined by one all-gather per step" % (WORKLOAD, n_sets_job, world),
                           "n_sets": n_sets_job, "paths_per_set": args.paths,
                           "n_steps": 16, "m": 7, "T": T, "weights": weights_kind,
                           "l2": "flushed between timed steps (256 MB write, outside the events)",
                           "parallelism": "dp%d" % world},
                "roofline": roof, "clocks": clk.summary(), "gpu_launches": launches_per_step * args.steps,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": n_e2e, "pipeline": "result copy of step k on a copy stream overlaps step k+1"},
                "cpu_baseline": cpu, "accuracy": accuracy, "kernel_ms": k_ms, "autotune": tuning,
                "secondary": secondary}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
