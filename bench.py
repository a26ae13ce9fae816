"""Benchmark of the vectorised CHIP-8 environment step on GB300.

Default workload (N = 1): the largest single-GPU configuration, 262,144
instances of 64 seeded random-opcode ROMs (3,584 B each, CXNN at 10 %),
K = 10 instructions per frame, frame skip 4, uint8 [4,32,64] observation
stack; K timed env steps (default 2,000 = the whole workload) from the
freshly reset state. ``--config scale|batch|schip|shooter|wrappers|small``
selects the other workloads.

One JSON line on stdout (rank 0). ``value`` is whole-job env steps/s with the
actions already in HBM, through octax_step_n (CUDA-graph replay, launch
configuration from octax_autotune); ``plain_kernel`` is the same workload with
one plain kernel launch per env step; ``e2e`` goes through octax_step_host
with pinned host buffers (actions in, obs/reward/done out, every step).
``--impl reference`` times the CPU oracle (the plain-C reference interpreter)
on the host cores instead. Multi-GPU runs are independent replicas (the
environments never exchange data); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_01764_gb300 import workloads as W  # noqa: E402

METRIC = "env steps/s on 1 GB300 (bit-exact vs oracle) vs plain kernel; serving p50/p99 ms"

# Algorithmic HBM bytes of the step kernel. Per env step and instance: the
# observation (4 frames) + action + reward + done. Per launch and instance:
# the emulator state read at the start and written at the end (V 16, PC|I 4,
# SP|timers|status 4, stack 32, display, dirty mask 8, counters 8, previous
# score 4, previous action 1; read only: Philox key 8, uid 4, output row 4;
# SCHIP adds the mode byte).
def frame_shape(w: W.Workload) -> tuple:
    return (64, 128) if w.games[0].variant == "schip" else (32, 64)


def step_io_bytes(w: W.Workload) -> int:
    r, c = frame_shape(w)
    return 4 * r * c + 1 + 4 + 1


def state_bytes(w: W.Workload) -> int:
    schip = w.games[0].variant == "schip"
    disp = 1024 if schip else 256
    # V, PC|I, SP|timers|status, stack, display, page mask, written-address
    # range, counters, previous score and action, SCHIP mode byte
    written = 16 + 4 + 4 + 32 + disp + 8 + 4 + 8 + 4 + 1 + (1 if schip else 0)
    return written + (written + 16)  # written, and read back with the 16 read-only bytes


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(values: list, device=None) -> list:
    """Element-wise maximum over all ranks (identity on one process). The
    environments never exchange data; this is only the timing reduction."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def step_plan(steps: int, rollout: int, warmup: int) -> dict:
    """How the K timed env steps are cut into octax_step_n calls.

    T (the rollout ring's depth, the autotuner's call length) is at most the
    step count, so a short run (``--steps 20``) tunes and times 20-step calls
    rather than asking for more action rows than it generated. ``calls`` are
    the [lo, hi) step ranges of the timed region (T steps each, the last one
    ragged); ``warmup`` are the untimed step indices replayed before it (at
    least one, cycling through the K action rows), followed by the first
    calls again so that every graph the timed region replays exists."""
    if steps < 1:
        raise ValueError("need at least one timed step")
    T = max(1, min(rollout, steps))
    calls = [(lo, min(lo + T, steps)) for lo in range(0, steps, T)]
    return {"T": T, "calls": calls, "warmup": [s % steps for s in range(max(warmup, 1))],
            "warmup_calls": calls[:2]}


# Output ring that the default rollout length may fill (observations, rewards
# and done flags of one octax_step_n call).
ROLLOUT_RING_BYTES = 36e9


def default_rollout(n_envs: int, io_bytes: int, budget: float = ROLLOUT_RING_BYTES) -> int:
    """Env steps per octax_step_n call when --rollout is not given: the
    longest power of two from 32 (the paper's PPO rollout, §4.1) up to 256
    whose output ring, n_envs x io_bytes per step, fits in ``budget``; never
    below 32. A launch lasts until its slowest warp is done, so longer calls
    (and the longer launches they allow) spread the stragglers' wait."""
    T = 32
    while T < 256 and 2 * T * n_envs * io_bytes <= budget:
        T *= 2
    return T


def whole_job_rate(world: int, n_envs: int, steps: int, ms: float) -> float:
    """Env steps/s of the whole job: every replica ran n_envs x steps."""
    return world * n_envs * steps / (ms / 1e3)


def workload(name: str, n_envs: int = 0) -> W.Workload:
    """The named configuration; n_envs > 0 resizes it (profiling captures)."""
    make = {"scale": W.cfg_scale, "small": W.cfg_small, "batch": W.cfg_batch,
            "divergence": W.cfg_divergence, "schip": W.cfg_schip, "shooter": W.cfg_shooter,
            "wrappers": W.cfg_wrappers}[name]
    if n_envs > 0:
        if name == "small":
            raise SystemExit("--n-envs does not apply to the small configuration")
        return make(n_envs=n_envs)
    return make()


def describe(config: str, w: W.Workload) -> str:
    g = w.games[0]
    return {
        "scale": f"plain-scale: {w.n_envs} instances of the template ROM (seed 2, {len(g.rom)} B), "
                 "K=10, frameskip 4, obs uint8 [4,32,64], auto-reset at score>=20 or 5,000 steps",
        "small": f"plain-small: {w.n_envs} instances of the template ROM (seed 1), K=10, frameskip 4",
        "batch": f"batch: {w.n_envs} instances over 16 template ROMs (200-3,000 B), K per ROM in "
                 "{5,8,10,15,20}, uneven episodes, 16 frames per persistent graph launch",
        "divergence": f"divergence: {w.n_envs} instances of 64 random-opcode ROMs (3,584 B), K=10",
        "schip": f"schip-scale: {w.n_envs} instances of the hires Super-CHIP template ROM (seed 3, "
                 f"{len(g.rom)} B), K=20, frameskip 4, obs uint8 [4,64,128], auto-reset at score>=20 "
                 "or 2,000 steps",
        "wrappers": f"wrappers: the plain-scale workload ({w.n_envs} template instances, K=10, frameskip 4) "
                    "with sticky actions (p = 0.25) and no-op resets (0-30 steps)",
        "shooter": f"target-shooter: {w.n_envs} instances of the Target Shooter levels 1-3 (one third each, "
                   f"{'/'.join(str(len(x.rom)) for x in w.games)} B), K=10, frameskip 4, uniform random "
                   "actions over 5, auto-reset after 10 targets or 5,000 steps",
    }[config]


def data_kind(config: str) -> str:
    return {"divergence": "synthetic (seeded random-opcode ROMs, Philox actions)",
            "shooter": "Target Shooter ROMs (written from the paper's description), Philox actions",
            }.get(config, "synthetic (seeded template ROMs, Philox actions)")


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def strip_comments(src: str) -> str:
    """C/C++ source without comments and with whitespace collapsed (string
    literals in the kernel sources hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash() -> str:
    """Hash of the step kernel's code (comments and layout ignored), which ties
    a recorded ncu traffic figure to the code it was measured on."""
    h = hashlib.sha256()
    for f in ("octax_kernels.cu", "octax_internal.h"):
        h.update(strip_comments(open(os.path.join(ROOT, "paper_2510_01764_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(config: str) -> dict | None:
    """Per-instance-step DRAM bytes and warp instructions of the step kernel
    from the committed ncu summary, if it was taken on the current kernel
    source (otherwise None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(config)
    if not e or e.get("kernel_source") != kernel_source_hash():
        return None
    return e


_NCU_SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-9, "ns": 1e-9,
              "usecond": 1e-6, "us": 1e-6, "msecond": 1e-3, "ms": 1e-3, "second": 1.0, "s": 1.0}


def record_traffic(csv_path: str, config: str, launch: str, units: int, n_envs: int = 0) -> dict:
    """Store the step kernel's DRAM bytes and warp instructions per instance
    step, averaged over the launches of an `ncu --page raw --csv` export, in
    profiles/traffic.json under `config` (tagged with the kernel source hash)."""
    import csv

    rows = list(csv.reader(open(csv_path)))
    hdr, unit_row, data = rows[0], rows[1], [r for r in rows[2:] if r and "step_kernel" in ",".join(r)]
    if not data:
        raise SystemExit(f"no step_kernel launch in {csv_path}")

    def mean(name: str) -> float:
        i = hdr.index(name)
        scale = _NCU_SCALE.get(unit_row[i], 1.0)
        return sum(float(r[i].replace(",", "")) for r in data) / len(data) * scale

    traffic = mean("dram__bytes_read.sum") + mean("dram__bytes_write.sum")
    entry = {
        "kernel_source": kernel_source_hash(),
        "captured_launch": launch,
        "captured_n_envs": n_envs or workload(config).n_envs,
        "captured_launches": len(data),
        "captured_instance_steps_per_launch": units,
        "dram_bytes_per_launch": traffic,
        "dram_bytes_per_instance_step": traffic / units,
        "warp_inst_per_instance_step": mean("smsp__inst_executed.sum") / units,
        "active_threads_per_warp_inst": mean("smsp__thread_inst_executed_per_inst_executed.ratio"),
        "branch_uniform_pct": mean("smsp__sass_average_branch_targets_threads_uniform.pct"),
        "captured_duration_s": mean("gpu__time_duration.sum"),
        "note": "ncu --set full --clock-control none; DRAM write bytes exclude observation "
                "lines still in L2 at kernel exit",
    }
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        d = {}
    d[config] = entry
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    return entry


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args) -> dict | None:
    import torch

    from paper_2510_01764_gb300 import octax

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    w = workload(args.config, args.n_envs)
    K, Wm = args.steps if args.steps else w.n_steps, args.warmup
    n = w.n_envs
    plan = step_plan(K, args.rollout or default_rollout(n, step_io_bytes(w)), Wm)
    T, calls = plan["T"], plan["calls"]
    with torch.cuda.stream(stream):
        env = octax.Env(w.games, n, seed=w.seed, quirks=w.quirks, game_of_env=w.game_of_env,
                        device=local, stream=stream)
        acts_h = W.actions(w.action_seed, 0, K, n, w.games[0].n_actions)
        acts = torch.from_numpy(acts_h).to(dev)
        obs = torch.empty((T, n, 4) + frame_shape(w), dtype=torch.uint8, device=dev)
        rew = torch.empty((T, n), dtype=torch.float32, device=dev)
        done = torch.empty((T, n), dtype=torch.uint8, device=dev)
        init_state = env.get_state()

        # ---- launch configuration: autotuned for T-step calls
        if args.launch:
            f = [int(x) for x in args.launch.split(",")] + [0, 0]
            env.set_launch(block=f[0], inst_per_warp=f[1], steps_per_launch=f[2], persistent=f[3],
                           use_graph=f[4], writer_warps=f[5], balance=f[6])
        else:
            env.autotune(T, acts[:T])
        launch = env.launch

        def run_calls(cfg: dict | None):
            if cfg:
                env.set_launch(**cfg)
            for lo, hi in calls:
                c = hi - lo
                env.step_n(acts[lo:hi], out=(obs[:c], rew[:c], done[:c]))

        def timed(cfg: dict | None) -> tuple[float, int]:
            # warm-up (graph build, caches) then restore the fresh state
            if cfg:
                env.set_launch(**cfg)
            for s in plan["warmup"]:
                env.step_n(acts[s:s + 1], out=(obs[:1], rew[:1], done[:1]))
            for lo, hi in plan["warmup_calls"]:
                env.step_n(acts[lo:hi], out=(obs[:hi - lo], rew[:hi - lo], done[:hi - lo]))
            env.set_state(init_state)
            torch.cuda.synchronize(dev)
            if world > 1:
                torch.distributed.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_calls(None)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            dn = int(done.sum().item())
            return ms, dn

        with Clocks(local) as clk:
            ms_best, _ = timed(launch)
        clocks = clk.summary()
        plain_cfg = dict(block=launch["block"], inst_per_warp=launch["inst_per_warp"],
                         steps_per_launch=1, persistent=0, use_graph=0, writer_warps=0, balance=0)
        ms_plain, _ = timed(plain_cfg)
        env.set_launch(**launch)

        # ---- the same calls writing bit-packed observations (octax_step_n_packed)
        pobs = torch.empty((T, n) + env.packed_obs_shape, dtype=torch.int64, device=dev)
        for lo, hi in plan["warmup_calls"]:
            env.step_n_packed(acts[lo:hi], out=(pobs[:hi - lo], rew[:hi - lo], done[:hi - lo]))
        env.set_state(init_state)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for lo, hi in calls:
            env.step_n_packed(acts[lo:hi], out=(pobs[:hi - lo], rew[:hi - lo], done[:hi - lo]))
        p1.record(stream)
        torch.cuda.synchronize(dev)
        ms_packed = p0.elapsed_time(p1)
        del pobs

        # ---- end to end through the host-buffer entry point
        Ke = min(K, args.e2e_steps)
        a_h = torch.from_numpy(acts_h[:Ke].copy()).pin_memory()
        o_h = torch.empty((n, 4) + frame_shape(w), dtype=torch.uint8, pin_memory=True)
        r_h = torch.empty(n, dtype=torch.float32, pin_memory=True)
        d_h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        env.set_launch(**plain_cfg)
        for s in range(min(3, Ke)):
            env.step_host(a_h[s], out=(o_h, r_h, d_h))
        env.set_state(init_state)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for s in range(Ke):
            env.step_host(a_h[s], out=(o_h, r_h, d_h))
        e2e_s = time.perf_counter() - t0
        # the same through the packed host-buffer entry point
        po_h = torch.empty((n,) + env.packed_obs_shape, dtype=torch.int64, pin_memory=True)
        env.set_state(init_state)
        for s in range(min(3, Ke)):
            env.step_host_packed(a_h[s], out=(po_h, r_h, d_h))
        env.set_state(init_state)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for s in range(Ke):
            env.step_host_packed(a_h[s], out=(po_h, r_h, d_h))
        e2e_packed_s = time.perf_counter() - t0
        env.set_launch(**launch)

    ms_best, ms_plain, e2e_s, ms_packed, e2e_packed_s = max_over_ranks(
        [ms_best, ms_plain, e2e_s, ms_packed, e2e_packed_s], dev)
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        return None

    value = whole_job_rate(world, n, K, ms_best)
    spl = launch["steps_per_launch"]
    n_launch = sum((hi - lo + spl - 1) // spl for lo, hi in calls)
    launch_ms = ms_best / n_launch
    alg_bytes = n * (step_io_bytes(w) * (K / n_launch) + state_bytes(w))
    peak, peak_src = measured_peaks()
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    prof = profiled_traffic(args.config)
    units_per_launch = n * K / n_launch
    traffic = None if prof is None else round(prof["dram_bytes_per_instance_step"] * units_per_launch)
    issue = None
    if prof is not None and clocks.get("sm_mhz"):
        import torch as _t
        sms = _t.cuda.get_device_properties(dev).multi_processor_count
        peak_issue = sms * 4 * clocks["sm_mhz"] * 1e6          # warp-instructions/s
        got = prof["warp_inst_per_instance_step"] * units_per_launch / (launch_ms / 1e3)
        issue = {"achieved": round(got / 1e9, 2), "peak": round(peak_issue / 1e9, 2),
                 "unit": "G warp-instr/s", "frac": round(got / peak_issue, 4),
                 "divergence_efficiency": (round(prof["active_threads_per_warp_inst"] / 32, 4)
                                           if "active_threads_per_warp_inst" in prof else None),
                 "branch_efficiency": (round(prof["branch_uniform_pct"] / 100, 4)
                                       if "branch_uniform_pct" in prof else None),
                 "source": "ncu instruction count per instance-step (profiles/traffic.json) x "
                           "instance-steps per launch / live launch time; peak = SMs x 4 x median SM clock"}
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "env steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": round(ms_best / K, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": data_kind(args.config),
        "frames_per_s": round(value * w.games[0].frameskip, 1),
        "config": {
            "workload": describe(args.config, w),
            "n_envs_per_gpu": n,
            "steps": K,
            "rollout_buffer_steps": T,
            "launch": launch,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": (f"no flush: each step writes {n * (step_io_bytes(w) - 6) / 1e6:.0f} MB of observations "
                   f"into a {T}-step rollout ring ({T * n * (step_io_bytes(w) - 6) / 1e6:.0f} MB); "
                   f"emulator state {n * (state_bytes(w) / 2 + 4096) / 1e6:.0f} MB; L2 126 MB"),
        },
        "plain_kernel": {
            "value": round(whole_job_rate(world, n, K, ms_plain), 1),
            "unit": "env steps/s",
            "ms_per_step": round(ms_plain / K, 6),
            "launch": plain_cfg,
        },
        "speedup_vs_plain": round(ms_plain / ms_best, 3),
        "packed_obs": {
            "value": round(whole_job_rate(world, n, K, ms_packed), 1),
            "unit": "env steps/s",
            "ms_per_step": round(ms_packed / K, 6),
            "obs_bytes_per_env_step": (step_io_bytes(w) - 6) // 8,
            "hbm_frac": round(n * (((step_io_bytes(w) - 6) // 8 + 6) * (K / n_launch) + state_bytes(w))
                              / (ms_packed / n_launch / 1e3) / 1e9 / peak, 4),
            "e2e": {"value": round(world * n * Ke / e2e_packed_s, 1), "unit": "env steps/s", "steps": Ke,
                    "h2d_bytes_per_step": n,
                    "d2h_bytes_per_step": n * ((step_io_bytes(w) - 6) // 8 + 5),
                    "entry": "octax_step_host_packed"},
            "note": "octax_step_n_packed, same workload and launch: one bit per pixel (u64 row words)",
        },
        "gpu_launches": n_launch,
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "peak_source": peak_src,
            "kernel": "step_kernel",
            "bytes_per_launch": int(alg_bytes),
            "launch_ms": round(launch_ms, 5),
            "traffic": traffic,
            "traffic_source": None if prof is None else
            "ncu dram__bytes_read+write per instance-step (profiles/traffic.json) scaled to this launch",
        },
        "issue_roofline": issue,
        "e2e": {
            "value": round(world * n * Ke / e2e_s, 1),
            "unit": "env steps/s",
            "steps": Ke,
            "h2d_bytes_per_step": n,
            "d2h_bytes_per_step": n * (step_io_bytes(w) - 1),
        },
        "clocks": clocks,
    }
    if not args.no_policy and world == 1:
        line["policy"] = run_policy(args, dev, stream)
    if not args.no_serve and world == 1:
        line["serving"] = run_serving(args, dev)
        line["serving_p50_ms"] = line["serving"]["poisson"]["x1"]["p50_ms"]
        line["serving_p99_ms"] = line["serving"]["poisson"]["x1"]["p99_ms"]
    return line


# --------------------------------------------------------------------------- policy
def policy_flops(n_logits: int) -> int:
    """Algorithmic FLOPs (2 per multiply-add) of the §4.1 network per
    instance: conv1 15x15x32 outputs of 4x8x4 inputs, conv2 6x6x64 of
    32x4x4, conv3 4x4x64 of 64x3x3, the two 1024 -> 256 hidden layers and the
    256 -> n_logits / 256 -> 1 output layers."""
    conv = 15 * 15 * 32 * 128 + 6 * 6 * 64 * 512 + 4 * 4 * 64 * 576
    heads = 1024 * 512 + 256 * (n_logits + 1)
    return 2 * (conv + heads)


def policy_computed_flops(n_logits: int) -> int:
    """FLOPs the tensor cores execute per instance, including the rows of
    positions outside each layer's output (the kernels' tap-shift tiling):
    conv1 14 tiles, conv2 3 tiles, conv3 2 tiles of 128 rows per 8
    instances, heads 128-row tiles."""
    conv = (14 * 128 * 32 * 128 + 3 * 128 * 64 * 512 + 2 * 128 * 64 * 576) / 8
    return int(2 * (conv + 1024 * 512 + 256 * (n_logits + 1)))


def pack_words(obs):
    """uint8 frames [..., 32, 64] (0/1) -> int64 words [..., 32], bit x = pixel x."""
    import torch

    return (obs.to(torch.int64) << torch.arange(64, device=obs.device)).sum(dim=-1)


def run_policy(args, dev, stream) -> dict:
    """The §4.1 network acting in the environment on the device: the fused
    rollout (octax_rollout_policy: packed frames handed to the network
    through an L2-resident ring) against the environment step writing uint8
    observations to HBM followed by a separate network forward on them, and
    the network forward alone against the tensor roofline."""
    import torch

    from paper_2510_01764_gb300 import octax

    w = W.cfg_scale(n_envs=args.policy_envs)
    g = w.games[0]
    n, L, T = w.n_envs, g.n_actions + 1, args.policy_steps
    params = W.policy_params(1, L)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    with torch.cuda.stream(stream):
        env = octax.Env(w.games, n, seed=w.seed, device=dev.index, stream=stream)
        pol = octax.Policy(params, max_envs=n, device=dev.index, stream=stream)
        obs0 = env.reset()
        env.autotune(1)  # both legs step the environment one step per call
        words0 = pack_words(obs0)
        init = env.get_state()
        outs = (torch.empty((T, n), dtype=torch.uint8, device=dev),
                torch.empty((T, n, L), dtype=torch.float32, device=dev),
                torch.empty((T, n), dtype=torch.float32, device=dev),
                torch.empty((T, n), dtype=torch.float32, device=dev),
                torch.empty((T, n), dtype=torch.uint8, device=dev))

        def fused(steps):
            words = words0.clone()
            env.set_state(init)
            torch.cuda.synchronize(dev)
            e0, e1 = ev(), ev()
            e0.record(stream)
            pol.rollout(env, steps, words, seed=1, out=tuple(o[:steps] for o in outs))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1)

        obs = torch.empty_like(obs0)
        lg = torch.empty((n, L), dtype=torch.float32, device=dev)
        val = torch.empty(n, dtype=torch.float32, device=dev)
        act = torch.empty(n, dtype=torch.uint8, device=dev)

        def separate(steps):
            obs.copy_(obs0)
            env.set_state(init)
            torch.cuda.synchronize(dev)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for k in range(steps):
                pol.forward_u8(obs, seed=1, step=k, out=(lg, val, act))
                env.step(act, out=(obs, outs[3][k], outs[4][k]))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1)

        def forward_only(reps):
            torch.cuda.synchronize(dev)
            e0, e1 = ev(), ev()
            e0.record(stream)
            for k in range(reps):
                pol.forward(words0, seed=1, step=k, out=(lg, val, act))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1) / reps

        for _ in range(2):
            fused(min(T, 4))
            separate(min(T, 4))
            forward_only(3)
        ms_fused = min(fused(T) for _ in range(2))
        ms_sep = min(separate(T) for _ in range(2))
        ms_fwd = min(forward_only(max(4, T // 2)) for _ in range(2))
        pol.sync()
        env.set_state(init)
        del env, pol
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    fl = policy_flops(L)
    achieved = fl * n / (ms_fwd / 1e3) / 1e12
    return {
        "workload": f"{n} instances of the template ROM (seed 2), K=10, frameskip 4; the §4.1 network "
                    f"(convolutions 32/64/64, heads 256) with {L} logits, seeded random weights",
        "n_envs": n, "steps": T,
        "fused_rollout": {"value": round(n * T / (ms_fused / 1e3), 1), "unit": "env steps/s",
                          "ms_per_step": round(ms_fused / T, 5),
                          "entry": "octax_rollout_policy (packed frames through an L2-resident ring)"},
        "env_step_plus_separate_forward": {
            "value": round(n * T / (ms_sep / 1e3), 1), "unit": "env steps/s", "ms_per_step": round(ms_sep / T, 5),
            "entry": "octax_step (uint8 observations to HBM) + octax_policy_forward_u8 per step"},
        "speedup_fused": round(ms_sep / ms_fused, 3),
        "forward_ms": round(ms_fwd, 5),
        "roofline": {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "peak_source": "measured bf16 burst (cuBLAS)",
                     "kernels": "policy_conv_kernel + policy_heads_kernel (one forward)",
                     "flops_per_instance": fl, "computed_flops_per_instance": policy_computed_flops(L)},
    }


# --------------------------------------------------------------------------- serving
SERVE_RATES = (10.0, 100.0, 1000.0)   # requests/s per game, games cycle through the three


def serving_requests(n_req: int, seed: int, rate_scale: float = 1.0) -> dict:
    """n_req requests of the serving configuration: per game Poisson
    arrivals at 10, 100 or 1000 requests/s (times rate_scale), envs
    log-uniform in 1..4096, 1-8 steps, seeds; as arrays, sorted by arrival."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    rates = np.array([SERVE_RATES[g % 3] for g in range(16)]) * rate_scale
    # per-game arrival processes merged: game of each arrival ~ rate share, gaps ~ exponential(total rate)
    game = rng.choice(16, size=n_req, p=rates / rates.sum()).astype(np.uint16)
    t = np.cumsum(rng.exponential(1.0 / rates.sum(), size=n_req))
    envs = np.clip(np.rint(np.exp(rng.uniform(0.0, np.log(4096.0), size=n_req))), 1, 4096).astype(np.int64)
    steps = rng.integers(1, 9, size=n_req).astype(np.int64)
    seeds = rng.integers(0, 2 ** 62, size=n_req, dtype=np.int64).astype(np.uint64)
    return {"t": t - t[0], "game": game, "envs": envs, "steps": steps, "seed": seeds}


def _requests_for(srv, rq, sel, acts, act_off, obs, rew, done, out_off):
    """REQUEST_DTYPE rows for requests `sel`: actions from the flat host array
    at act_off, outputs from the flat device buffers at out_off (env-steps)."""
    r = np.zeros(len(sel), dtype=srv.REQUEST_DTYPE)
    r["game"], r["n_envs"], r["n_steps"] = rq["game"][sel], rq["envs"][sel], rq["steps"][sel]
    r["seed"] = rq["seed"][sel]
    r["actions"] = acts.ctypes.data + act_off
    o = out_off.astype(np.uint64)
    r["obs"] = np.uint64(obs.data_ptr()) + o * np.uint64(8192)
    r["reward"] = np.uint64(rew.data_ptr()) + o * np.uint64(4)
    r["done"] = np.uint64(done.data_ptr()) + o
    return r


def run_serving(args, dev) -> dict:
    """The serving configuration (16 template ROMs of the batch workload;
    requests of 1-4,096 envs and 1-8 steps): the server's launch shape chosen
    by measurement, a saturated closed-loop run of at least
    --serve-sat-steps env steps, open-loop Poisson arrivals at three offered
    loads, and octax_step_n on the same 16 ROMs for comparison."""
    import torch

    from paper_2510_01764_gb300 import octax

    games = W.cfg_batch(n_envs=64, n_steps=1).games
    budget = int(args.serve_budget_gb * 1e9)
    big = serving_requests(200_000, 55)
    ES = big["envs"] * big["steps"]
    act_h = np.random.Generator(np.random.Philox(key=56)).integers(0, 4, size=int(ES.sum()), dtype=np.uint8)
    act_off = np.concatenate([[0], np.cumsum(ES)[:-1]])
    half = int(args.serve_ring_steps)                      # env-steps of outputs per ring half
    obs = torch.empty((2 * half, 4, 32, 64), dtype=torch.uint8, device=dev)
    rew = torch.empty(2 * half, dtype=torch.float32, device=dev)
    done = torch.empty(2 * half, dtype=torch.uint8, device=dev)

    def saturated(block, ipw, min_steps):
        """Requests of the stream in waves, each wave filling one half of the
        output ring; a half is reused once its previous wave is done."""
        srv = octax.Server(games, memory_budget_bytes=budget, block=block, inst_per_warp=ipw,
                           max_inflight_ticks=2, device=dev.index)
        pending = [None, None]
        lat, first, last, steps, k, h = [], None, None, 0, 0, 0
        while steps < min_steps:
            if pending[h] is not None:
                inf = srv.wait_raw(pending[h])
                lat.append(inf[:, 2] - inf[:, 0])
                last = max(last or 0, int(inf[:, 2].max()))
            cum = np.cumsum(ES[k:k + 4096])
            m = int(np.searchsorted(cum, half, side="right"))
            sel = np.arange(k, k + m)
            if k + m >= len(ES):
                break
            out_off = h * half + np.concatenate([[0], cum[:m - 1]])
            ids = srv.submit_raw(_requests_for(srv, big, sel, act_h, act_off[sel], obs, rew, done, out_off))
            first = first or time.monotonic_ns()
            pending[h] = ids
            steps += int(cum[m - 1])
            k += m
            h ^= 1
        for hh in (0, 1):
            if pending[hh] is not None:
                inf = srv.wait_raw(pending[hh])
                lat.append(inf[:, 2] - inf[:, 0])
                last = max(last or 0, int(inf[:, 2].max()))
        srv.close()
        lat = np.concatenate(lat) / 1e6
        return steps / ((last - first) / 1e9), lat, steps, k

    # launch shape by measurement (short saturated runs)
    shapes = {}
    for block, ipw in ((64, 8), (128, 8), (128, 16), (256, 8), (256, 16)):
        saturated(block, ipw, 2 * half)                       # warm-up (graphs, caches)
        shapes[f"{block}x{ipw}"] = saturated(block, ipw, 8 * half)[0]
    best = max(shapes, key=shapes.get)
    bb, bi = (int(x) for x in best.split("x"))
    rate, lat, steps, nreq = saturated(bb, bi, args.serve_sat_steps)
    sat = {"env_steps": steps, "requests": nreq, "env_steps_per_s": round(rate, 1),
           "p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4),
           "latency_note": "closed loop: each wave of requests fills one half of a "
                           f"{2 * half * 8192 / 1e9:.1f} GB output ring and waits for the wave before it; "
                           "latency = done - submit, so it includes the wave's own queueing"}

    # open-loop Poisson arrivals at three offered loads
    poisson = {}
    for scale in (1.0, 5.0, 15.0):
        rq = serving_requests(100_000, 57, rate_scale=scale)
        es = rq["envs"] * rq["steps"]
        n_req = int(np.searchsorted(np.cumsum(es), args.serve_steps)) + 1
        cum = np.concatenate([[0], np.cumsum(es[:n_req])])
        if cum[-1] > 2 * half:
            n_req = int(np.searchsorted(cum, 2 * half, side="right")) - 1
        aoff = np.concatenate([[0], np.cumsum(es[:n_req])[:-1]])
        srv = octax.Server(games, memory_budget_bytes=budget, block=bb, inst_per_warp=bi, max_inflight_ticks=2,
                           device=dev.index)
        warm = srv.submit_raw(_requests_for(srv, rq, np.arange(16), act_h, aoff[:16], obs, rew, done, aoff[:16]))
        srv.wait_raw(warm)
        all_ids, sched, i = [], [], 0
        t0 = time.monotonic_ns()
        while i < n_req:
            now = (time.monotonic_ns() - t0) / 1e9
            j = int(np.searchsorted(rq["t"][:n_req], now, side="right"))
            if j > i:
                sel = np.arange(i, j)
                all_ids.append(srv.submit_raw(_requests_for(srv, rq, sel, act_h, aoff[sel], obs, rew, done,
                                                            aoff[sel])))
                sched.append(t0 + (rq["t"][sel] * 1e9).astype(np.int64))
                i = j
        inf = srv.wait_raw(np.concatenate(all_ids))
        srv.close()
        sched = np.concatenate(sched)
        lat = (inf[:, 2] - sched) / 1e6                     # from the scheduled arrival
        lat_srv = (inf[:, 2] - inf[:, 0]) / 1e6             # from the submit call
        span = (inf[:, 2].max() - sched.min()) / 1e9
        offered = cum[n_req] / max(rq["t"][n_req - 1], 1e-9)
        poisson[f"x{scale:g}"] = {
            "offered_env_steps_per_s": round(float(offered), 1), "requests": n_req,
            "env_steps": int(cum[n_req]), "env_steps_per_s": round(float(cum[n_req] / span), 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "server_p50_ms": round(float(np.percentile(lat_srv, 50)), 4),
            "server_p99_ms": round(float(np.percentile(lat_srv, 99)), 4)}

    # octax_step_n on the same 16 ROMs: the batch workload's 65,536 instances
    w = W.cfg_batch()
    env = octax.Env(w.games, w.n_envs, seed=w.seed, game_of_env=w.game_of_env, device=dev.index)
    a = torch.from_numpy(W.actions(w.action_seed, 0, 32, w.n_envs, 4)).to(dev)
    env.autotune(32, a)
    o2 = torch.empty((32, w.n_envs, 4, 32, 64), dtype=torch.uint8, device=dev)
    r2 = torch.empty((32, w.n_envs), dtype=torch.float32, device=dev)
    d2 = torch.empty((32, w.n_envs), dtype=torch.uint8, device=dev)
    env.step_n(a, out=(o2, r2, d2))
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cs = torch.cuda.current_stream(dev)
    e0.record(cs)
    for _ in range(2):
        env.step_n(a, out=(o2, r2, d2))
    e1.record(cs)
    torch.cuda.synchronize(dev)
    step_n_rate = 2 * 32 * w.n_envs / (e0.elapsed_time(e1) / 1e3)
    del env, o2, r2, d2, obs, rew, done
    torch.cuda.empty_cache()
    return {"games": 16, "budget_gb": args.serve_budget_gb,
            "requests": "per game Poisson 10/100/1000 requests/s (x the offered-load scale); envs "
                        "log-uniform 1-4096; 1-8 steps; uniform actions over 4",
            "launch_shapes_env_steps_per_s": {k: round(v, 1) for k, v in shapes.items()},
            "launch": {"block": bb, "inst_per_warp": bi},
            "saturated": sat, "poisson": poisson,
            "step_n_same_roms": {"env_steps_per_s": round(step_n_rate, 1), "n_envs": w.n_envs,
                                 "launch": "autotuned, 32-step calls"}}


# --------------------------------------------------------------------------- CPU oracle
def cpu_oracle(w: W.Workload, budget_s: float, threads: int, steps_hint: int | None = None) -> dict:
    import oracle

    oracle.build()
    n = w.n_envs
    env = oracle.OracleEnv(w.games, n, seed=w.seed, quirks=w.quirks, game_of_env=w.game_of_env)
    env.reset()
    acts = W.actions(w.action_seed, 0, 3, n, w.games[0].n_actions)
    t0 = time.perf_counter()
    env.step(acts[0], threads=threads)
    per_step = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(per_step, 1e-6)))
    if steps_hint:
        steps = min(steps, steps_hint)
    acts = W.actions(w.action_seed, 1, 1 + steps, n, w.games[0].n_actions)
    t0 = time.perf_counter()
    for s in range(steps):
        env.step(acts[s], threads=threads)
    dt = time.perf_counter() - t0
    return {"value": round(n * steps / dt, 1), "unit": "env steps/s", "cores": threads,
            "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"{n} instances x {steps} steps of the same workload (obs materialised)"}


def run_reference_rank_gate() -> bool:
    """The reference arm runs on rank 0 only; other ranks exit without work."""
    return dist_env()[0] == 0


def run_reference(args) -> dict | None:
    rank, world, _ = dist_env()
    if not run_reference_rank_gate():
        return None
    w = workload(args.config, args.n_envs)
    threads = os.cpu_count() or 1
    K, Wm = args.steps if args.steps else w.n_steps, args.warmup
    import oracle

    oracle.build()
    # each step: one env step over a bounded sample of the instances, sized so
    # that warm-up + K steps take about args.ref_budget seconds
    probe = oracle.OracleEnv(w.games, min(w.n_envs, 4096), seed=w.seed,
                             game_of_env=None if w.game_of_env is None else w.game_of_env[:4096])
    a = W.actions(w.action_seed, 0, 2, probe.n, w.games[0].n_actions)
    probe.step(a[0], threads=threads)
    t0 = time.perf_counter()
    probe.step(a[1], threads=threads)
    rate = probe.n / (time.perf_counter() - t0)
    probe.close()
    m = int(max(64, min(w.n_envs, rate * args.ref_budget / max(1, K + Wm))))
    goe = None if w.game_of_env is None else w.game_of_env[:m]
    env = oracle.OracleEnv(w.games, m, seed=w.seed, game_of_env=goe)
    env.reset()
    for s in range(Wm):
        env.step(W.actions(w.action_seed, s, s + 1, m, w.games[0].n_actions)[0], threads=threads)
    acts = W.actions(w.action_seed, 0, K, m, w.games[0].n_actions) if K * m <= 2e9 else None
    t0 = time.perf_counter()
    for s in range(K):
        row = acts[s] if acts is not None else W.actions(w.action_seed, s, s + 1, m, w.games[0].n_actions)[0]
        env.step(row, threads=threads)
    dt = time.perf_counter() - t0
    value = m * K / dt
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "env steps/s",
            "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": round(dt * 1e3 / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": data_kind(args.config),
            "config": {"workload": describe(args.config, w), "n_envs_sampled": m},
            "cpu_baseline": {"value": round(value, 1), "unit": "env steps/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{m} of {w.n_envs} instances per step, {K} steps"},
            "e2e": {"value": round(value, 1), "unit": "env steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed env steps (0 = the workload's)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="octax", choices=["octax", "reference"])
    ap.add_argument("--config", default="divergence",
                    choices=["scale", "small", "batch", "divergence", "schip", "shooter", "wrappers"])
    ap.add_argument("--rollout", type=int, default=0,
                    help="steps per octax_step_n call (0 = the longest of 32..256 whose output "
                         "ring fits in 36 GB)")
    ap.add_argument("--n-envs", type=int, default=0,
                    help="resize the configuration (0 = its own size); for small profiling captures")
    ap.add_argument("--launch", default="",
                    help="block,inst_per_warp,steps_per_launch,persistent,graph[,writer_warps[,balance]] "
                         "(default: autotune)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=90.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-policy", action="store_true")
    ap.add_argument("--policy-envs", type=int, default=16384)
    ap.add_argument("--policy-steps", type=int, default=32)
    ap.add_argument("--serve-steps", type=int, default=1_000_000)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-sat-steps", type=int, default=60_000_000,
                    help="env steps of the saturated serving run")
    ap.add_argument("--serve-ring-steps", type=int, default=500_000,
                    help="env steps of outputs per half of the serving output ring")
    ap.add_argument("--record-traffic", default="", metavar="CSV",
                    help="no GPU: read an `ncu -i <rep> --page raw --csv` export of step_kernel "
                         "launches into profiles/traffic.json for --config")
    ap.add_argument("--traffic-launch", default="", help="launch string of the captured run")
    ap.add_argument("--traffic-units", type=int, default=0,
                    help="instance steps per captured launch (instances x steps per launch)")
    return ap.parse_args(argv)


def main():
    args = parse_args()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic, args.config, args.traffic_launch,
                                        args.traffic_units, args.n_envs), indent=1))
        return
    if args.impl == "reference":
        line = run_reference(args)
        if line:
            print(json.dumps(line), flush=True)
        return
    line = run_gpu(args)
    if line is None:
        return
    if not args.no_cpu and line["n_gpus"] == 1:
        w = workload(args.config, args.n_envs)
        line["cpu_baseline"] = cpu_oracle(w, args.cpu_budget, os.cpu_count() or 1)
        line["cpu_baseline"]["single_core"] = cpu_oracle(w, args.cpu_budget / 3, 1)["value"]
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
