#!/usr/bin/env python3
"""Throughput benchmark of the GB300 FNT-CDC + FNT-AEQ path.

One step = one pass of the whole hot path (FNT-CDC on both polarisations,
requantise + resample, FNT-AEQ with RDE adaptation) over one batch of synthetic
input already resident in device memory.  Default workload: one PDM-16QAM
stream, 40 GBaud at 2 samples/symbol, 2^20 symbols per polarisation, 75 km
(17 CD taps, 6 bit), 5-bit I/Q, AEQ 4x4 RV-MIMO at N = 64 / radix 4080 in
segments of 1024 symbols with 128 warm-up symbols, every segment starting from
the tap state the previous step ended with (a stream processed step by step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fnt|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (bounded sample of the same workload).  With N > 1 (launched
by torch.distributed.run) every rank runs an independent replica on its own GPU
(the path has no exchange step); value = all ranks' samples / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gsamples/s (PDM, 2 sps) bit-exact vs oracle"
UNIT = "Gsamples/s"

# ---------------------------------------------------------------- workload ----

WORKLOADS = {
    "cfg2": dict(n_sym=1 << 20, km=75.0, n_aeq=64, alpha_aeq=4080, segment=1024, warmup=128,
                 desc="PDM-16QAM 40 GBaud 2 sps, 2^20 symbols/pol (2^21 samples), 75 km, 17 CD taps (6 bit), "
                      "5-bit I/Q, FNT-CDC N=64 alpha=4080 S=48 + FNT-AEQ 4x4 RV-MIMO N=64 alpha=4080 K=16, "
                      "AEQ segments of 1024 symbols + 128 warm-up starting from the stream's carried taps"),
    "cfg5": dict(n_sym=1 << 26, km=80.0, n_aeq=32, alpha_aeq=2, segment=1 << 16, warmup=1 << 12,
                 desc="PDM bandwidth stress, 2^27 samples/pol, 80 km, 19 CD taps, FNT-AEQ N=32 alpha=2, "
                      "segments 2^16 + 2^12 warm-up"),
}
MU_SHIFT = 9
TAP_INIT = 2048

# Algorithmic integer-op model (one count per operation the method needs, at
# its cheapest: a Z_F radix-2 butterfly = add, subtract, twiddle multiply and
# one split-and-subtract reduction (shift + multiply-add) plus an amortised
# lazy reduction of the sum = 6; a pointwise product mod F = multiply +
# reduction = 3; an int64 gradient multiply-accumulate = 2).
OPS_BUTTERFLY, OPS_MULMOD, OPS_MAC = 6, 3, 2


def butterflies(n: int) -> int:
    return (n // 2) * int(math.log2(n))


def cdc_ops(n_samples: int, S: int, n_pol: int = 2) -> float:
    """Per polarisation and block: 2 forward + 2 inverse FNT-64, 2 x 64 products."""
    blocks = math.ceil(n_samples / S)
    return n_pol * blocks * (4 * butterflies(64) * OPS_BUTTERFLY + 2 * 64 * OPS_MULMOD)


def aeq_ops(n_sym: int, na: int) -> float:
    """Per block of na - 16 symbols: 4 input + 32 tap + 32 inverse FNT-na,
    32 x na products, 16 x 16 x (na - 16) gradient MACs."""
    sa = na - 16
    per_block = 68 * butterflies(na) * OPS_BUTTERFLY + 32 * na * OPS_MULMOD + 16 * 16 * sa * OPS_MAC
    return n_sym / sa * per_block


def alu_peak_ops() -> float:
    """Issue-bound INT32 peak: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz."""
    return 152 * 4 * 32 * 2070e6


def source_hash(*names: str) -> str:
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2405_04253_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, src_hash: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; otherwise None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != src_hash:
        return None
    return rec.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ clocks ----

class ClockSampler:
    """nvidia-smi samples (100 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.rows = []
        self.proc = None
        if gpu_id is None:
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({self.NAMES[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------- multi-rank ----

def reduce_max(x: float, device=None) -> float:
    """Max of a float over the ranks of the default process group (identity
    without one).  Used for timings only; the data path has no collective."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(samples_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput in Gsamples/s: every rank's samples over the slowest
    rank's time (weak scaling: each rank runs its own replica)."""
    return world * samples_per_rank / max_seconds / 1e9


# ----------------------------------------------------------------- oracle ----

_W = {}


def _worker_init(x, taps, prm_kw, T0):
    import oracle
    oracle.build()
    _W.update(x=x, taps=taps, prm=oracle.ChainParams(**prm_kw), T0=T0)


def _worker_noop(i):
    return i


def _worker_segment(seg):
    import oracle
    keep, out, _ = oracle.chain_segment(_W["x"], _W["taps"], _W["prm"], seg, T0=_W["T0"])
    return seg, keep, out


class OraclePool:
    """Spawned worker processes holding the stream once each; a run over a set
    of AEQ segments is timed from submission to the last result (start-up
    excluded)."""

    def __init__(self, x, taps, prm_kw, procs, T0):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_worker_init,
                                                 initargs=(x, taps, prm_kw, T0))
        self.pool.map(_worker_noop, range(procs), chunksize=1)

    def run(self, segs):
        t0 = time.perf_counter()
        res = {s: (k, o) for s, k, o in self.pool.imap_unordered(_worker_segment, segs, chunksize=1)}
        secs = time.perf_counter() - t0
        samples = sum(2 * o.shape[0] for (_, o) in res.values())
        return secs, samples, res

    def close(self):
        self.pool.close()
        self.pool.join()


def _prm_kw(wl):
    return dict(n_aeq=wl["n_aeq"], alpha_aeq=wl["alpha_aeq"], mu_shift=MU_SHIFT, seg_len=wl["segment"],
                warmup=wl["warmup"])


def _segments(x_np, taps, wl, n_seg):
    L = taps.shape[0]
    nsym = (x_np.shape[0] - (((L - 1) // 2) & 1) + 1) // 2
    total = math.ceil(nsym / wl["segment"])
    return sorted({int(i * total / n_seg) for i in range(n_seg)}), total


# ---------------------------------------------------------------- main arm ----

def run_fnt(args, rank, world, local_rank):
    import torch
    import paper_2405_04253_gb300 as fnt
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = WORKLOADS[args.workload]
    gen = synth.config2 if args.workload == "cfg2" else synth.config5
    frame = gen(wl["n_sym"]) if args.workload == "cfg2" else synth.config5(2 * wl["n_sym"])
    x_np, taps = frame.x, frame.taps
    n = x_np.shape[0]
    L = taps.shape[0]
    S = 64 - L + 1
    plan = fnt.Plan(n_aeq=wl["n_aeq"], alpha_aeq=wl["alpha_aeq"], mu_shift=MU_SHIFT,
                    aeq_segment=wl["segment"], aeq_warmup=wl["warmup"])
    nsym = fnt.chain_nsym(n, L)
    x = torch.from_numpy(x_np).to(dev)
    out = torch.zeros((nsym, 4), dtype=torch.int16, device=dev)
    state = torch.zeros((4, 4, 16), dtype=torch.int32, device=dev)       # the stream's carried AEQ taps
    state[[0, 1, 2, 3], [0, 1, 2, 3], 8] = TAP_INIT << 16
    batch = fnt.Batch(plan, [fnt.Frame(x, out, taps, state)], fnt.OP_CHAIN, use_graph=False)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        batch.launch_stage(0, stream)
        if evs:
            evs[1].record(stream)
        batch.launch_stage(1, stream)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    clocks = ClockSampler(gpu_id if rank == 0 else None)
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (outside the events)
        step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    cdc_ms = [e[0].elapsed_time(e[1]) for e in evs]
    aeq_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = reduce_max(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = aggregate(n, world, ms_per_step * 1e-3)

    # one more step from a recorded tap state: its output is what the CPU-baseline
    # leg recomputes on sampled segments
    state_snap = state.cpu().numpy().copy()
    step()
    torch.cuda.synchronize()
    out_check = out.clone()

    # end to end through the public call with host buffers (pinned), copies included
    e2e = None
    if args.e2e_steps > 0:
        xh = torch.from_numpy(x_np).pin_memory()
        oh = torch.empty((nsym, 4), dtype=torch.int16).pin_memory()
        st_e2e = torch.from_numpy(state_snap).to(dev)
        fr = [fnt.Frame(xh, oh, taps, st_e2e)]
        fnt.cdc_aeq_run(plan, fr, host=True)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fnt.cdc_aeq_run(plan, fr, host=True)
        el = reduce_max(time.perf_counter() - t0, dev)
        e2e = {"value": aggregate(n * args.e2e_steps, world, el), "unit": UNIT,
               "h2d_bytes_per_step": int(x_np.nbytes), "d2h_bytes_per_step": int(oh.numel() * 2),
               "ms_per_step": el / args.e2e_steps * 1e3, "api": "fnt_cdc_aeq_run(host_buffers=1)"}
        st_e2e.copy_(torch.from_numpy(state_snap))
        fnt.cdc_aeq_run(plan, fr, host=True)
        e2e["bitexact_vs_device_path"] = bool(torch.equal(oh, out_check.cpu()))

    # roofline of the dominant kernel
    aeq_avg = statistics.mean(aeq_ms)
    cdc_avg = statistics.mean(cdc_ms)
    dom = "aeq" if aeq_avg >= cdc_avg else "cdc"
    ops = aeq_ops(nsym, wl["n_aeq"]) if dom == "aeq" else cdc_ops(n, S)
    dur = aeq_avg if dom == "aeq" else cdc_avg
    kname = f"aeq_kernel<{wl['n_aeq']}>" if dom == "aeq" else "cdc_kernel<chain>"
    src = source_hash("aeq.cu", "zf.cuh", "internal.h") if dom == "aeq" else source_hash("cdc.cu", "zf.cuh",
                                                                                      "internal.h")
    achieved = ops / (dur * 1e-3) / 1e12
    peak = alu_peak_ops() / 1e12
    roof = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 3), "peak": round(peak, 2),
            "unit": "Tops/s (int32, algorithmic)", "frac": round(achieved / peak, 4),
            "traffic": profiled_traffic(kname, src), "avg_launch_ms": round(dur, 4),
            "peak_basis": "152 SMs x 4 schedulers x 32 lanes x 2070 MHz (issue-bound int32)"}
    hbm_bytes = n * 4 + nsym * 8
    res = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "samples_per_step": n, "symbols_per_step": nsym,
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "aeq_mu_shift": MU_SHIFT, "rde_a": 64},
        "roofline": roof,
        "kernels_ms": {"cdc": round(cdc_avg, 4), "aeq": round(aeq_avg, 4)},
        "hbm": {"achieved_gbs": round(hbm_bytes / (ms_per_step * 1e-3) / 1e9, 2), "peak_gbs": 6795.1,
                "frac": round(hbm_bytes / (ms_per_step * 1e-3) / 1e9 / 6795.1, 5),
                "bytes_per_step": hbm_bytes, "note": "algorithmic: int8 input + int16 output"},
        "gpu_launches": args.steps * batch.kernel_count(),
        "clocks": clk,
        "wall_s_timed_region": round(wall, 3),
        "e2e": e2e,
    }
    return res, (x_np, taps, out_check, wl, state_snap)


def init_taps():
    T = np.zeros((4, 4, 16), np.int32)
    for s_ in range(4):
        T[s_, s_, 8] = TAP_INIT << 16
    return T


def cpu_baseline(x_np, taps, wl, out_dev=None, n_seg=96, procs=None, T0=None):
    """The oracle as it stands on a bounded sample: n_seg AEQ segments spread
    over the stream, in a spawn pool over the host cores."""
    procs = procs or min(os.cpu_count() or 1, n_seg)
    segs, total = _segments(x_np, taps, wl, n_seg)
    pool = OraclePool(x_np, taps, _prm_kw(wl), procs, init_taps() if T0 is None else T0)
    try:
        secs, samples, res = pool.run(segs)
    finally:
        pool.close()
    cb = {"value": round(samples / secs / 1e9, 6), "unit": UNIT, "cores": procs, "kind": "oracle",
          "sample": f"{len(segs)} of {total} AEQ segments ({samples} output samples) of the same stream, plain C "
                    f"oracle (O(N^2) transforms), spawn pool", "seconds": round(secs, 2)}
    if out_dev is not None:
        got = out_dev.cpu().numpy()
        cb["sample_bitexact"] = bool(all(np.array_equal(got[k:k + o.shape[0]], o) for (k, o) in res.values()))
    return cb


def run_reference(args):
    """The CPU oracle as the reference arm: each step a bounded sample of the
    same workload (args.ref_segments AEQ segments) on the host cores."""
    import synth
    wl = WORKLOADS[args.workload]
    frame = synth.config2(wl["n_sym"]) if args.workload == "cfg2" else synth.config5(2 * wl["n_sym"])
    procs = min(os.cpu_count() or 1, 16)
    segs, total = _segments(frame.x, frame.taps, wl, args.ref_segments)
    pool = OraclePool(frame.x, frame.taps, _prm_kw(wl), procs, init_taps())
    try:
        for _ in range(args.warmup):
            pool.run(segs[:procs])
        secs, samples = 0.0, 0
        for _ in range(args.steps):
            s_, n_, _ = pool.run(segs)
            secs += s_
            samples += n_
    finally:
        pool.close()
    value = samples / secs / 1e9
    sample = f"{len(segs)} of {total} AEQ segments per step, plain C oracle (O(N^2) transforms), spawn pool"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload + ": " + wl["desc"], "samples_per_step": samples // args.steps},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["fnt", "reference"], default="fnt")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg2")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-segments", type=int, default=128)
    ap.add_argument("--ref-segments", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res, (x_np, taps, out, wl, T0) = run_fnt(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(x_np, taps, wl, out, n_seg=args.cpu_segments, T0=T0)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
