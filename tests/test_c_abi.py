"""The C-ABI used from C alone: tests/c_abi_rollout.c includes only
include/octax.h, links liboctax.so and steps with host buffers. The CPU test
compiles it against the header; the GPU test runs it and compares its
per-instance state hashes, reward and done totals with the CPU oracle."""
import os
import subprocess

import numpy as np
import pytest

from paper_2510_01764_gb300 import workloads as W
from paper_2510_01764_gb300.workloads import Clause, GameSpec, Term

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_rollout.c")
INC = os.path.join(ROOT, "include")


def test_c_program_compiles_against_the_header(tmp_path):
    obj = tmp_path / "c_abi_rollout.o"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", INC, "-c", SRC,
                           "-o", str(obj)])


@pytest.mark.gpu
@pytest.mark.parametrize("packed", [False, True])
def test_c_program_matches_oracle(tmp_path, packed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2510_01764_gb300 import build

    lib = build.build()
    oracle.build()
    exe = tmp_path / "c_abi_rollout"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-I", INC, SRC, "-o", str(exe),
                           "-L", os.path.dirname(lib), "-loctax",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    rom = W.template_rom(W.TemplateParams(seed=6, deco_pairs=1))
    rom_path = tmp_path / "game.ch8"
    rom_path.write_bytes(rom)
    n, steps, seed = 77, 300, 12345
    out = subprocess.run([str(exe), str(rom_path), str(n), str(steps), str(seed)] + (["packed"] if packed else []),
                         capture_output=True, text=True, check=True).stdout.split("\n")
    got = [int(line, 16) for line in out[:n]]
    summary = out[n].split()

    game = GameSpec(rom=rom, instr_per_frame=10, frameskip=4, stack_frames=4, action_set=(7, 9, 5, 8),
                    score=(Term("reg", 6),), term=(Clause(Term("reg", 6), ">=", 3),))
    ref = oracle.OracleEnv([game], n, seed=seed)
    ref.reset()
    i = np.arange(n)
    reward_sum, done_sum = 0.0, 0
    for s in range(steps):
        o, r, d = ref.step(((7 * i + 3 * s) % 5).astype(np.uint8), obs=s == steps - 1)
        reward_sum += float(r.sum())
        done_sum += int(d.sum())
    assert got == [int(h) for h in ref.hashes()]
    assert summary == ["reward", f"{reward_sum:.0f}", "done", str(done_sum), "lit", str(int(o.sum()))]
    assert done_sum > 0
