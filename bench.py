"""Benchmark: progressive refactoring + retrieval on one GB300 per rank.

One step = the whole hot path over one 512^3 FP32 field (a seeded Gaussian
random field with P(k) ~ k^-11/3, rescaled to [-1, 1]): refactor once, then six
incremental retrievals at relative L-infinity bounds 1e-1 .. 1e-6 on the same
handle.  Throughput follows the paper's definition (Sec. 7.2.2: bytes of the
original data for refactoring, of the reconstructed data for retrieval), so
one step moves 7 x 512 MiB of field bytes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank refactors its own
field (replicas: the method exchanges nothing between sub-domains) and the
value is the sum over ranks of the field bytes divided by the slowest rank's
time.  `--impl reference` times the plain CPU oracle on a bounded sub-block of
the same field on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("refactor & retrieve GB/s (1 GB300) and % HBM roofline; served p50/p99 retrieval "
          "latency")
TAUS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
WORKLOAD = ("512^3 FP32 spectral field (P(k)~k^-11/3, rescaled to [-1,1], seed 2 + rank): "
            "refactor + 6 incremental retrievals at relative Linf 1e-1..1e-6")
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ fields
def make_field(n, seed, device):
    import torch
    from paper_2505_00227_gb300 import synthetic
    return synthetic.spectral((n, n, n), seed=seed, dtype=torch.float32, device=device)


def traffic_for(kernel):
    """DRAM bytes per launch from a committed ncu capture of the same kernel
    source, or None when there is none or the source changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            table = json.load(fh)
        e = table[kernel]
        src = os.path.join(ROOT, "paper_2505_00227_gb300", "csrc", e["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != e["source_sha256"]:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------- CPU oracle
def oracle_step(f_np):
    from oracle import pyoracle as O
    t0 = time.perf_counter()
    F = O.Field(f_np)
    for tau in TAUS:
        F.retrieve(tau * F.range)  # each retrieval of the oracle starts from the stored bytes
    return time.perf_counter() - t0


def cpu_baseline(field_dev, side):
    import numpy as np
    sub = field_dev[:side, :side, :side].contiguous().cpu().numpy()
    t = oracle_step(np.ascontiguousarray(sub))
    gbs = 7 * sub.nbytes / t / 1e9
    return {"value": round(gbs, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"one step (refactor + 6 retrievals) on the [0:{side}]^3 sub-block of the "
                      f"same 512^3 field, single-threaded C oracle, {t:.2f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    field = make_field(args.size, 2, dev)
    side = args.ref_side
    import numpy as np
    sub = np.ascontiguousarray(field[:side, :side, :side].contiguous().cpu().numpy())
    del field
    for _ in range(args.warmup):
        oracle_step(sub)
    times = [oracle_step(sub) for _ in range(args.steps)]
    total = sum(times)
    value = 7 * sub.nbytes * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"[0:{side}]^3 sub-block per step"},
        "cpu_baseline": {"value": round(value, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"[0:{side}]^3 sub-block of the 512^3 field, refactor + 6 "
                                   "retrievals per step, single-threaded C oracle"},
        "e2e": {"value": round(value, 6), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_00227_gb300 import binding

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.size
    field = make_field(n, 2 + rank, "cuda")
    N = field.numel()
    fbytes = N * field.element_size()
    ctx = binding.Context()
    out = torch.empty_like(field)
    stream = torch.cuda.current_stream()

    def step(rec=None):
        h = ctx.refactor(field)
        if rec is not None:
            rec.append(torch.cuda.Event(enable_timing=True))
            rec[-1].record(stream)
        infos = []
        for tau in TAUS:
            _, info, st = h.retrieve(tau, out=out)
            infos.append(info)
        h.free()
        return infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region (value, roofline) ----------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.profile(True)
    launches0 = binding.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    marks = []
    starts = []
    t_start.record(stream)
    last_infos = None
    for _ in range(args.steps):
        starts.append(torch.cuda.Event(enable_timing=True))
        starts[-1].record(stream)
        last_infos = step(marks)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = binding.kernel_launches() - launches0
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    refactor_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(starts, marks))
    retrieve_ms = ms - refactor_ms
    prof = ctx.profile_entries()
    ctx.profile(False)

    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    step_bytes = 7 * fbytes
    value = world * step_bytes / (ms_max * 1e-3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers ---------
    host_in = field.cpu().pin_memory()
    host_out = torch.empty(field.shape, dtype=field.dtype).pin_memory()

    def step_host():
        h = ctx.refactor(host_in)
        for tau in TAUS:
            h.retrieve(tau, out=host_out)
        h.free()

    step_host()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_t = torch.tensor([e2e_s], device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * step_bytes / float(e2e_t.item()) / 1e9

    if rank == 0:
        peak, peak_kind = peaks()
        stages = [p for p in prof if p[2] > 0]
        total_ms = sum(p[1] for p in stages) or 1.0
        dominant = max((p for p in stages if p[3] > 0), key=lambda p: p[1])
        name, kms, calls, kbytes = dominant
        achieved = kbytes / (kms * 1e-3) / 1e9
        traffic = traffic_for(name)
        roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "algorithmic_bytes_per_launch": kbytes / calls,
                "avg_launch_ms": kms / calls,
                "traffic": traffic}
        kernels = [{"stage": p[0], "launches_per_step": p[2] / args.steps,
                    "ms_per_step": round(p[1] / args.steps, 4), "share": round(p[1] / total_ms, 4),
                    "gbs": round(p[3] / (p[1] * 1e-3) / 1e9, 1) if p[3] > 0 and p[1] > 0 else None}
                   for p in sorted(stages, key=lambda p: -p[1])]
        fetched = [i.bytes_fetched_total for i in last_infos]
        alg_refactor = fbytes  # the field is read once; stored bytes are written below
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(field, args.cpu_side)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "field_bytes": fbytes, "step_bytes": step_bytes,
                       "l2": "inputs larger than L2 (512 MiB per field)",
                       "parallelism": f"replicas x{world}"},
            "refactor_gbs": round(fbytes / (refactor_ms * 1e-3) / 1e9, 3),
            "retrieve_gbs": round(6 * fbytes / (retrieve_ms * 1e-3) / 1e9, 3),
            "refactor_ms": round(refactor_ms, 4), "retrieve_ms": round(retrieve_ms, 4),
            "retrieved_bytes_total": fetched, "roofline": roof, "kernels": kernels,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": "GB/s", "h2d_bytes_per_step": fbytes,
                    "d2h_bytes_per_step": 6 * fbytes},
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--cpu-side", type=int, default=256)
    ap.add_argument("--ref-side", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
