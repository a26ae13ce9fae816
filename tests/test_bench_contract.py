"""bench.py's output contract and bookkeeping, without a GPU: the reference
arm's JSON line (the CPU oracle on the host cores), the algorithmic byte
counts behind the roofline, the workload descriptions, and how ncu exports
become per-instance-step traffic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2510_01764_gb300 import workloads as W  # noqa: E402

BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
             "scaling", "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--config", "small", "--steps", "3", "--warmup", "3", "--ref-budget", "1"],
                         capture_output=True, text=True, check=True, cwd=ROOT, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "env steps/s"
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("name", ["scale", "small", "batch", "divergence", "schip", "shooter", "wrappers"])
def test_workload_descriptions_and_bytes(name):
    w = bench.workload(name)
    text = bench.describe(name, w)
    assert str(w.n_envs) in text
    schip = w.games[0].variant == "schip"
    assert bench.frame_shape(w) == ((64, 128) if schip else (32, 64))
    # observation stack + action + reward + done per env step
    assert bench.step_io_bytes(w) == 4 * (8192 if schip else 2048) + 6
    # state written back and read again per launch (display 1 KB for SCHIP)
    assert bench.state_bytes(w) == (2228 if schip else 690)
    assert bench.data_kind(name)


def test_workload_resize():
    assert bench.workload("divergence", 65536).n_envs == 65536
    with pytest.raises(SystemExit):
        bench.workload("small", 10)


def test_record_traffic_from_an_ncu_export(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "feedface")
    cols = ["Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum",
            "smsp__thread_inst_executed_per_inst_executed.ratio",
            "smsp__sass_average_branch_targets_threads_uniform.pct", "gpu__time_duration.sum"]
    units = ["", "Mbyte", "Gbyte", "inst", "", "%", "us"]
    row = ["void step_kernel_chip8<1>(StepLaunch)", "8", "4", "655360", "9.5", "90", "800"]
    csv_path = tmp_path / "raw.csv"
    csv_path.write_text("\n".join(",".join(f'"{c}"' for c in r) for r in (cols, units, row)) + "\n")
    e = bench.record_traffic(str(csv_path), "scale", "256,7,32,0,1,0,1", 1000)
    assert e["kernel_source"] == "feedface" and e["captured_n_envs"] == 16384
    assert e["dram_bytes_per_launch"] == pytest.approx(8e6 + 4e9)
    assert e["dram_bytes_per_instance_step"] == pytest.approx((8e6 + 4e9) / 1000)
    assert e["warp_inst_per_instance_step"] == pytest.approx(655.36)
    assert e["captured_duration_s"] == pytest.approx(800e-6)
    stored = json.load(open(tmp_path / "profiles" / "traffic.json"))
    assert stored["scale"] == e
    assert bench.profiled_traffic("scale") == e          # same source hash: used
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.profiled_traffic("scale") is None       # kernel changed: not used


def test_kernel_source_hash_ignores_comments():
    a = "int f() { return 1; } // one\n/* block */\n"
    b = "int f() {   return 1; }\n"
    assert bench.strip_comments(a).split() == bench.strip_comments(b).split()


@pytest.mark.parametrize("steps,warmup,rollout", [(20, 5, 32), (1, 3, 32), (33, 3, 32), (2000, 3, 32),
                                                  (64, 0, 32), (7, 9, 4)])
def test_step_plan(steps, warmup, rollout):
    """The timed calls cover exactly steps 0..K-1 in order, each at most T
    long, T never exceeds K (the autotuner and the rollout ring are sized
    from T), and every warm-up index is a valid action row."""
    p = bench.step_plan(steps, rollout, warmup)
    T = p["T"]
    assert 1 <= T <= min(rollout, steps)
    assert p["calls"][0][0] == 0 and p["calls"][-1][1] == steps
    for (lo, hi), (lo2, _) in zip(p["calls"], p["calls"][1:]):
        assert hi == lo2
    assert all(0 < hi - lo <= T for lo, hi in p["calls"])
    assert len(p["warmup"]) == max(warmup, 1) and all(0 <= s < steps for s in p["warmup"])
    assert p["warmup_calls"] == p["calls"][:2]


def test_default_rollout_by_workload():
    """With no --rollout, each configuration gets the longest power-of-two
    rollout from 32 to 256 whose output ring fits the 36 GB budget: the
    16,384-instance CHIP-8 workloads 256 steps, the 65,536-instance batch and
    the Super-CHIP workload (4x larger frames) 64, the 262,144-instance
    default 32; the driver's 20-step command still times one 20-step call."""
    rings = {}
    for name, T_want in [("scale", 256), ("wrappers", 256), ("shooter", 256), ("small", 256),
                         ("schip", 64), ("batch", 64), ("divergence", 32)]:
        w = bench.workload(name)
        io = bench.step_io_bytes(w)
        T = bench.default_rollout(w.n_envs, io)
        assert T == T_want, name
        assert T == 32 or T * w.n_envs * io <= bench.ROLLOUT_RING_BYTES
        rings[name] = T * w.n_envs * io
    assert max(rings.values()) < 70e9  # the 32-step floor at 262,144 instances
    w = bench.workload("divergence")
    p = bench.step_plan(20, bench.default_rollout(w.n_envs, bench.step_io_bytes(w)), 5)
    assert p["T"] == 20 and p["calls"] == [(0, 20)]
    assert bench.default_rollout(1, 1) == 256 and bench.default_rollout(10**9, 10**4) == 32
    assert bench.parse_args([]).rollout == 0


def test_step_plan_driver_command():
    """A short run (--steps 20 --warmup 5) tunes and times one 20-step call;
    the default run (2,000 steps) uses 32-step calls."""
    p = bench.step_plan(20, 32, 5)
    assert p["T"] == 20 and p["calls"] == [(0, 20)]
    p = bench.step_plan(2000, 32, 3)
    assert p["T"] == 32 and len(p["calls"]) == 63 and p["calls"][-1] == (1984, 2000)
    p = bench.step_plan(33, 32, 3)
    assert p["calls"] == [(0, 32), (32, 33)]
    with pytest.raises(ValueError):
        bench.step_plan(0, 32, 3)


def test_default_config_is_the_largest_single_gpu_workload():
    a = bench.parse_args(["--gpus", "1", "--steps", "20", "--warmup", "5"])
    assert a.config == "divergence" and a.steps == 20 and a.warmup == 5
    assert bench.workload(a.config).n_envs == 262144


def test_policy_flop_counts():
    """§4.1 layer sizes: conv1 15x15x32 of 4x8x4, conv2 6x6x64 of 32x4x4,
    conv3 4x4x64 of 64x3x3, heads 1024 -> 2 x 256 and 256 -> L / 256 -> 1."""
    macs = 15 * 15 * 32 * 128 + 6 * 6 * 64 * 512 + 4 * 4 * 64 * 576 + 1024 * 512 + 256 * 6
    assert bench.policy_flops(5) == 2 * macs == 6433792
    # the tap-shift tiling executes more (dropped rows, zero halves of conv1's stacked weights)
    assert bench.policy_computed_flops(5) > bench.policy_flops(5)


def test_pack_words_matches_packbits():
    torch = pytest.importorskip("torch")
    import numpy as np

    obs = (np.random.default_rng(0).random((3, 4, 32, 64)) < 0.3).astype(np.uint8)
    want = np.packbits(obs, axis=-1, bitorder="little").view("<u8").reshape(3, 4, 32).view(np.int64)
    got = bench.pack_words(torch.from_numpy(obs)).numpy()
    assert np.array_equal(got, want)


def test_serving_request_stream():
    """Arrivals sorted from 0, games weighted by their rates (10/100/1000 per
    s, cycling), envs in 1..4096 (log-uniform), steps in 1..8, rate scaling
    shortens the gaps."""
    import numpy as np

    rq = bench.serving_requests(20000, 55)
    assert rq["t"][0] == 0 and np.all(np.diff(rq["t"]) >= 0)
    assert rq["envs"].min() >= 1 and rq["envs"].max() <= 4096
    assert set(np.unique(rq["steps"])) == set(range(1, 9))
    counts = np.bincount(rq["game"], minlength=16)
    fast = [g for g in range(16) if g % 3 == 2]
    slow = [g for g in range(16) if g % 3 == 0]
    assert counts[fast].min() > 20 * counts[slow].max()
    # log-uniform sizes: about as many below 64 as above
    assert 0.35 < (rq["envs"] < 64).mean() < 0.65
    fast_rq = bench.serving_requests(20000, 55, rate_scale=15.0)
    assert fast_rq["t"][-1] == pytest.approx(rq["t"][-1] / 15.0, rel=1e-9)
