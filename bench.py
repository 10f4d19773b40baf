#!/usr/bin/env python
"""Throughput of the qEW explicit-Euler relaxation (arXiv:1211.7275, Sec. II-III) on GB300.

Metric: site-updates/s = sum over chains of L x Euler steps, divided by the device time of the
relaxation.  One bench step is one full pass of the hot path over the workload: reset to the flat
start, integrate `relax_steps` Euler steps with the fused FP32-split kernel, record v and w2 at
log-spaced observation steps (fused reductions) and bring them to the host.

Default workload: 4 random-field chains of L = 2^25 (the paper's largest size, Sec. IV.D), dt = 0.1,
drive at the preset's critical force.  The 4 GiB state is larger than the 129 MB L2, so no flush
is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead (the baseline arm).
Under torchrun (N > 1) each rank relaxes its own independent samples (weak scaling, no collective
on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import qew_workloads as W  # noqa: E402

METRIC = "site-updates/s and % binding roofline, qEW Euler at L=2^25, FP32-split vs FP64, 1 GB300"
UNIT = "site-updates/s"

# Algorithmic lane operations per site-update of the fused kernel, per disorder kind (0 RF,
# 1 uniform RB cubic, 2 none, 3 Gaussian RB linear, 4 Gaussian RB cubic): elastic force 6,
# pinning 2 (linear) / 8 (cubic) / 0 (none), Euler 3, renormalisation and cell test 3; plus, per
# cell crossing, one Philox4x32-10 block (~90 integer operations with its key schedule) and the
# value transform (Box-Muller ~13, uniform ~2).
OPS_BASE = {0: 14, 1: 20, 2: 12, 3: 14, 4: 20}
OPS_PER_CROSSING = {0: 103, 1: 92, 2: 0, 3: 103, 4: 103}
QUAD_KINDS = (1, 4)
LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="rf_4x2^25", choices=["rf_4x2^25", "rf_16x2^20", "rb_1024x2^16",
                                                                "rbg_linear_4x2^25", "none_16x2^20",
                                                                "uneven_256", "tiny_rf_1x1024"])
    p.add_argument("--relax-steps", type=int, default=4096)
    p.add_argument("--n-obs", type=int, default=12)
    p.add_argument("--tuning", default="auto", help="'auto' or tile_w,K,tiles_per_cta")
    p.add_argument("--fp64-steps", type=int, default=256, help="Euler steps of the FP64 comparison leg (0: skip)")
    p.add_argument("--horizon-steps", type=int, default=None,
                   help="Euler steps of the one relaxation timed at the workload's own horizon, outside the timed "
                        "loop (default: the preset's n_steps, 2^20 for rf_4x2^25; 0: skip)")
    p.add_argument("--horizon-obs", type=int, default=None, help="observations of that relaxation (default: the preset's)")
    p.add_argument("--others", default="rb_1024x2^16,uneven_256,rbg_linear_4x2^25,none_16x2^20",
                   help="presets whose fused kernels get a short roofline measurement beside the main line "
                        "(comma-separated; empty: none)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def rank_seed(rank: int) -> int:
    """Master seed of a rank: every rank relaxes its own independent disorder samples."""
    return W.SEED + 1000003 * rank


def workload(name: str, rank: int):
    """Chains of a preset: L, kind, f (scalars with ``batch`` chains, or per-chain arrays with
    batch None), the chain count, and the chain the CPU sample relaxes (``cpu``)."""
    p = W.PRESETS[name]
    if name == "uneven_256":
        n = p["n_chains"]
        L = W.uneven_lengths(n)
        kind = W.uneven_kinds(n)
        base = np.where(kind == W.RF, W.preset_f("rf_16x2^20"), W.preset_f("rb_1024x2^16"))
        f = base * (1.0 + W.sweep_offsets(n))
        c = int(np.argmax(L))
        return dict(name=name, L=L, batch=None, kind=kind, f=f, dt=p["dt"], seed=rank_seed(rank), n_chains=n,
                    cpu=dict(L=int(L[c]), batch=1, kind=int(kind[c]), f=float(f[c]), chain=c))
    return dict(name=name, L=p["L"], batch=p["batch"], kind=p["kind"], f=W.preset_f(name), dt=p["dt"],
                seed=rank_seed(rank), n_chains=p["batch"],
                cpu=dict(L=p["L"], batch=p["batch"], kind=p["kind"], f=W.preset_f(name), chain=0))


def describe(wl: dict) -> dict:
    """JSON-friendly shape of a workload."""
    if wl["batch"] is None:
        L = np.asarray(wl["L"])
        return {"L": f"{wl['n_chains']} chains, L from {int(L.min())} to {int(L.max())}, {int(L.sum())} sites",
                "kind": "mixed " + "/".join(str(k) for k in sorted(set(np.asarray(wl['kind']).tolist()))),
                "f": "per chain (f_c^L of its kind x (1 + {-2,-1,0,1,2}%))"}
    return {"L": wl["L"], "kind": wl["kind"], "f": wl["f"]}


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time is the slowest rank's (weak scaling: every rank does the same work)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def bus_id(dev: int) -> str | None:
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        return f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
    except Exception:
        return None


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("qew_split.cu", "qew_device.cuh", "qew_internal.h"):
        with open(os.path.join(ROOT, "paper_1211_7275_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per site per launch of the fused kernel, from the committed ncu summary, if it
    was captured on the current kernel source; else None.  Traffic is proportional to the sites a
    launch streams (not to K), so it scales to the bench's launches by their site count."""
    import re
    path = os.path.join(ROOT, "profiles", "split_step_kernel_rf_16x2e20.md")
    try:
        with open(path) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(r"traffic-record: kernel_sha=(\w+) dram_bytes_per_site_per_launch=([0-9.]+)", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    return float(m.group(2))


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline leg / reference arm)
# ------------------------------------------------------------------------------------------
def cpu_sample_shape(L: int) -> tuple[int, int]:
    """Window and steps of the CPU baseline sample: 2^20 sites x 128 steps per thread; chains
    shorter than 2^21 take half their length and proportionally more steps, within the light cone
    (w + 2 n <= L)."""
    w = min(1 << 20, L // 2)
    return w, min(128 * ((1 << 20) // w), (L - w) // 2)


def oracle_sample(wl: dict, w: int, n_steps: int) -> dict:
    """Time the CPU oracle on windows of the same chains: one light-cone window of w sites per host
    thread, n_steps Euler steps each (exact sites of the full-size chains)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cs = wl["cpu"]
    L = cs["L"]
    jobs = [(cs["chain"] if wl["batch"] is None else t % cs["batch"], (t * w * 7919) % L) for t in range(cores)]
    errs = []

    def work(c, i0):
        try:
            oracle.lightcone(L, c, cs["f"], wl["dt"], cs["kind"], wl["seed"], i0, w, min(n_steps, (L - w) // 2))
        except Exception as e:  # pragma: no cover
            errs.append(e)

    ths = [threading.Thread(target=work, args=j) for j in jobs]
    t0 = time.perf_counter()
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    dt = time.perf_counter() - t0
    if errs:
        raise errs[0]
    n_eff = min(n_steps, (L - w) // 2)
    updates = cores * w * n_eff
    return {"value": updates / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} threads x one light-cone window of {w} sites x {n_eff} Euler steps of the "
                      f"{wl['name']} chains (exact sites of the full-size chains), {dt:.1f} s",
            "seconds": dt}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    wl = workload(args.workload, 0)
    w, n = min(1 << 20, wl["cpu"]["L"] // 2), 48
    for _ in range(args.warmup):
        oracle_sample(wl, w, n)
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample(wl, w, n)
        vals.append(r["value"])
        secs.append(r["seconds"])
    cores = r["cores"]
    total = sum(cores * w * n for _ in vals)
    value = total / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], **describe(wl), "batch": wl["n_chains"],
                   "dt": wl["dt"], "arm": "CPU FP64 oracle (plain C, one light-cone window per host thread)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": r["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Launch shapes the autotuner picks for the other presets on a GB300 (their own relaxations, at
# step 1024); the short measurement below uses them directly instead of tuning again.
OTHER_SHAPES = {"rb_1024x2^16": (480, 16, 1), "uneven_256": (736, 32, 1), "rbg_linear_4x2^25": (480, 8, 1),
                "none_16x2^20": (736, 32, 2), "rf_16x2^20": (992, 32, 2), "rf_4x2^25": (992, 32, 2)}


def other_kernel(q, name: str, stream, sms: int, clk_mhz: float, n_steps: int = 1024) -> dict:
    """Site-updates/s and roofline fraction of the fused kernel on another preset: one relaxation of
    ``n_steps`` from the flat start in the preset's tuned shape (after one untimed run), fused
    observations at 12 log-spaced steps, device time from CUDA events on the library's stream."""
    import torch
    wl = workload(name, 0)
    sched = W.log_spaced_steps(n_steps, 12)
    r = q.Relaxation(wl["L"], wl["f"], wl["kind"], dt=wl["dt"], seed=wl["seed"], precision=q.FP32_SPLIT,
                     batch=wl["batch"], stream=stream)
    try:
        r.set_tuning(*OTHER_SHAPES[name])
        r.observe(sched)
        r.reset()
        r.enable_stats(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.observe(sched)
        e1.record(stream)
        torch.cuda.synchronize()
        st = r.stats()
        n_sites = r.n_sites
    finally:
        r.close()
    ms = e0.elapsed_time(e1)
    kinds = np.broadcast_to(np.asarray(wl["kind"]), (wl["n_chains"],))
    sites = np.broadcast_to(np.asarray(wl["L"], dtype=np.float64), (wl["n_chains"],))
    wk = {int(k): float(sites[kinds == k].sum() / sites.sum()) for k in set(kinds.tolist())}
    rx = st["crossings"] / max(1, st["site_updates"])
    ops = sum(w * (OPS_BASE[k] + OPS_PER_CROSSING[k] * rx) for k, w in wk.items())
    peak = sms * LANES_PER_SM * clk_mhz * 1e6 / 1e12
    ach = ops * st["site_updates"] / (st["fused_ms"] / 1e3) / 1e12 if st["fused_ms"] > 0 else None
    return {"value": n_sites * n_steps / (ms / 1e3), "unit": UNIT, "relax_steps": n_steps,
            "tuning": dict(zip(("tile_w", "K", "tiles_per_cta"), OTHER_SHAPES[name])),
            "crossings_per_site_update": rx, "ops_per_site_update": ops,
            "roofline_frac": (ach / peak) if ach else None, "fused_share": st["fused_ms"] / ms if ms > 0 else None}


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def main() -> None:
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1211_7275_gb300 as q

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    wl = workload(args.workload, rank)
    sched = W.log_spaced_steps(args.relax_steps, args.n_obs)
    # A stream of its own (torch's default stream has the null handle, which the library reads as
    # "use your own stream"): the kernels and the timing events then share one stream.
    stream = torch.cuda.Stream(device=local)
    relax = q.Relaxation(wl["L"], wl["f"], wl["kind"], dt=wl["dt"], seed=wl["seed"], precision=q.FP32_SPLIT,
                         batch=wl["batch"], stream=stream)
    if args.tuning == "auto":
        relax.set_tuning(0, 0, 0)
    else:
        relax.set_tuning(*[int(x) for x in args.tuning.split(",")])

    def one_step():
        relax.reset()
        relax.observe(sched)

    for _ in range(max(args.warmup, 3)):
        one_step()
    tuning = relax.tuning()

    sampler = ClockSampler(bus_id(local))
    relax.enable_stats(True)
    torch.cuda.synchronize()
    barrier()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        one_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    st = relax.stats()
    relax.enable_stats(False)
    n_sites = relax.n_sites
    updates = n_sites * args.relax_steps * args.steps
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(updates, world, ms_max)

    # ---- roofline of the fused kernel, from its own event-timed launches ----
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    per_launch_ms = st["fused_ms"] / max(1, st["fused_launches"])
    su_per_launch = st["site_updates"] / max(1, st["fused_launches"])
    r_cross = st["crossings"] / max(1, st["site_updates"])
    # per-kind figures weighted by the sites of each kind (one kind for every preset but the mixed batch)
    kinds = np.broadcast_to(np.asarray(wl["kind"]), (wl["n_chains"],))
    sites = np.broadcast_to(np.asarray(wl["L"], dtype=np.float64), (wl["n_chains"],))
    wk = {int(k): float(sites[kinds == k].sum() / sites.sum()) for k in set(kinds.tolist())}
    ops_per_su = sum(w * (OPS_BASE[k] + OPS_PER_CROSSING[k] * r_cross) for k, w in wk.items())
    achieved = ops_per_su * su_per_launch / (per_launch_ms / 1e3) / 1e12
    peak = sms * LANES_PER_SM * clk * 1e6 / 1e12
    tile_w, K, tpc = tuning
    bytes_per_su = sum(w * 2 * (8 + 4 * (6 if k in QUAD_KINDS else 2 if k != 2 else 0)) for k, w in wk.items()) / K
    hbm_achieved = bytes_per_su * su_per_launch / (per_launch_ms / 1e3) / 1e9
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    traffic = profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": (traffic * n_sites) if traffic else None,
                "kernel": "split_step_kernel (fused stencil+pinning+Euler+regeneration, K-step blocked)",
                "ops_per_site_update": ops_per_su, "crossings_per_site_update": r_cross,
                "per_launch_ms": per_launch_ms, "site_updates_per_launch": su_per_launch,
                "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes x {clk:.0f} MHz (median SM clock sampled "
                              "during the timed region)",
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                        "peak_basis": "MEASURED_PEAKS.json hbm_gbs (measured)"},
                "fused_share_of_step": st["fused_ms"] / ms if ms > 0 else None}

    # ---- measured lane-arithmetic rates (after the timed region): the peak above is derived from
    # unit counts and the sampled clock; this shows what the device sustains on plain FMA chains ----
    alu = q.measure_alu_peaks()
    roofline["alu_measured"] = {
        "fp32_fma_tops": alu["fp32_fma_per_s"] / 1e12, "sm_mhz": alu["sm_mhz"],
        "frac_of_measured_fp32_fma": achieved / (alu["fp32_fma_per_s"] / 1e12),
        "philox_blocks_per_s": alu["philox_blocks_per_s"],
        "regeneration_bound_su_per_s": alu["philox_blocks_per_s"] / r_cross if r_cross > 0 else None,
        "fp64_fma_tops": alu["fp64_fma_per_s"] / 1e12,
        "basis": "qew_measure_alu_peaks: best of 3 event-timed launches of independent FMA chains / Philox4x32-10 "
                 "blocks on a grid filling every SM"}

    # ---- one relaxation at the workload's own horizon (its preset's steps and observation count),
    # outside the timed loop: the crossing rate, and with it the speed, changes with t ----
    horizon = None
    h_steps = W.PRESETS[wl["name"]].get("n_steps", 0) if args.horizon_steps is None else args.horizon_steps
    if h_steps > 0:
        h_obs = args.horizon_obs or W.PRESETS[wl["name"]].get("n_obs", 100)
        hs = W.log_spaced_steps(h_steps, h_obs)
        split = min(h_steps, 1 << 16)   # the late part (steps past 2^16) is reported on its own
        parts = [hs[hs <= split], hs[hs > split]]
        relax.reset()
        relax.enable_stats(True)
        hsamp = ClockSampler(bus_id(local))
        torch.cuda.synchronize()
        hsamp.start()
        legs = []
        for part in parts:
            if part.size == 0:
                continue
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            relax.observe(part)
            e1.record(stream)
            torch.cuda.synchronize()
            hst = relax.stats()
            legs.append((e0.elapsed_time(e1), hst))
        hclk = hsamp.stop()
        relax.enable_stats(False)
        hpeak = sms * LANES_PER_SM * ((hclk or {}).get("sm_mhz") or clk) * 1e6 / 1e12

        def leg_fields(ms_leg, hst, steps):
            rx = hst["crossings"] / max(1, hst["site_updates"])
            ops = sum(w * (OPS_BASE[k] + OPS_PER_CROSSING[k] * rx) for k, w in wk.items())
            ach = ops * hst["site_updates"] / (hst["fused_ms"] / 1e3) / 1e12 if hst["fused_ms"] > 0 else None
            return {"steps": int(steps), "ms": ms_leg, "value": n_sites * steps / (ms_leg / 1e3),
                    "crossings_per_site_update": rx, "ops_per_site_update": ops,
                    "roofline_frac": (ach / hpeak) if ach else None,
                    "fused_share": hst["fused_ms"] / ms_leg if ms_leg > 0 else None}

        ms_h = sum(m for m, _ in legs)
        tot = {k: sum(h[k] for _, h in legs) for k in ("crossings", "site_updates", "fused_ms")}
        horizon = {"relax_steps": int(h_steps), "observations": int(hs.size), **leg_fields(ms_h, tot, h_steps),
                   "unit": UNIT, "peak": hpeak, "clocks": hclk,
                   "note": "one relaxation from the flat start, fused observations at the preset's log-spaced "
                           "steps, launch shape of the timed loop; value = site-updates / device time"}
        if len(legs) == 2:
            horizon["early"] = leg_fields(legs[0][0], legs[0][1], split)
            horizon["late"] = leg_fields(legs[1][0], legs[1][1], h_steps - split)

    # ---- the other presets' fused kernels: a short relaxation each, outside the timed region ----
    others = {}
    for name in [x for x in args.others.split(",") if x and x != wl["name"]]:
        others[name] = other_kernel(q, name, stream, sms, (clocks or {}).get("sm_mhz") or clk)

    # ---- structure factor (Eq. 6) of the relaxed chains, outside the timed region: the first call
    # builds the cuFFT plan; the second shows the steady state ----
    sq = None
    if len(set(np.atleast_1d(wl["L"]).tolist())) == 1:
        times = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S = relax.structure_factor()
            times.append(1e3 * (time.perf_counter() - t0))
        sq = {"ms_first": times[0], "ms": times[1], "modes": int(S.size), "chains": int(wl["n_chains"]),
              "includes": "state to FP64 rows, batched real-to-complex cuFFT, mean |u_q|^2 over chains, "
                          "copy to host (work area allocated and freed in the call); the first call also "
                          "builds the plan"}

    # ---- FP64 plain path on the same chains (the comparison the metric names) ----
    fp64 = None
    if args.fp64_steps > 0:
        relax.close()
        torch.cuda.synchronize()
        fs = W.log_spaced_steps(args.fp64_steps, 6)
        res = {}
        for prec, label in ((q.FP64, "fp64"), (q.FP32_SPLIT, "split")):
            r = q.Relaxation(wl["L"], wl["f"], wl["kind"], dt=wl["dt"], seed=wl["seed"], precision=prec,
                             batch=wl["batch"], stream=stream)
            if prec == q.FP32_SPLIT:
                r.set_tuning(*tuning)
            r.observe(fs)
            r.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                r.reset()
                r.observe(fs)
            e1.record(stream)
            torch.cuda.synchronize()
            res[label] = 2 * n_sites * args.fp64_steps / (e0.elapsed_time(e1) / 1e3)
            r.close()
        fp64 = {"value": res["fp64"], "split_same_window": res["split"], "relax_steps": args.fp64_steps,
                "split_over_fp64": res["split"] / res["fp64"]}
        relax = None

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        n_e2e = min(args.steps, 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            r = q.Relaxation(wl["L"], wl["f"], wl["kind"], dt=wl["dt"], seed=wl["seed"], precision=q.FP32_SPLIT,
                             batch=wl["batch"], stream=stream)
            r.set_tuning(*tuning)
            out = r.observe(sched)
            r.close()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        h2d = sched.nbytes + wl["n_chains"] * (8 + 8 + 4)
        d2h = len(sched) * wl["n_chains"] * 4 * 8
        e2e = {"value": n_sites * args.relax_steps * n_e2e / wall, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e,
               "includes": "handle creation (device allocation + flat-start init), relaxation with fused "
                           "observations, copy of the observables to host memory, destruction"}
        assert np.all(np.isfinite(out["v"]))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(wl, *cpu_sample_shape(wl["cpu"]["L"]))
        cpu.pop("seconds", None)

    state_gib = sum(w * (8 + 4 * (4 if k in QUAD_KINDS else 2 if k != 2 else 0)) for k, w in wk.items()) * n_sites / 2 ** 30
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], **describe(wl), "batch_per_gpu": wl["n_chains"],
                       "dt": wl["dt"], "relax_steps": args.relax_steps,
                       "observations": int(len(sched)), "precision": "int32 cell + f32 offset, f64 reductions",
                       "tuning": {"tile_w": tile_w, "K": K, "tiles_per_cta": tpc},
                       "l2": (f"inputs larger than L2 ({state_gib:.2f} GiB state), no flush" if state_gib > 0.129
                              else f"state of {state_gib * 1024:.1f} MiB fits in L2 (not a bandwidth measurement)"),
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": roofline, "horizon": horizon, "other_kernels": others or None, "fp64_path": fp64, "cpu_baseline": cpu, "e2e": e2e,
            "structure_factor": sq,
            "gpu_launches": st["launches"], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
