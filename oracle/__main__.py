"""Command line for the oracle (test infrastructure): run N instances of one
ROM for S steps with seeded actions and print, per step, the FNV-1a state hash
of every instance, then the summed reward and done counts.

    python -m oracle ROM --envs 4 --steps 10 [--seed 1] [--action-seed 1]
        [--actions 4] [--ipf 10] [--frameskip 4] [--score-reg 6] [--variant chip8]

Actions are the seeded Philox streams of paper_2510_01764_gb300.workloads
(index `--actions` is the no-op); the score is one register, so rewards are
its increases.
"""
import argparse

import numpy as np

import oracle
from paper_2510_01764_gb300 import workloads as W


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m oracle")
    ap.add_argument("rom")
    ap.add_argument("--envs", type=int, default=4)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--action-seed", type=int, default=1)
    ap.add_argument("--actions", type=int, default=4, help="action-set size (keys 7, 9, 5, 8, ...)")
    ap.add_argument("--ipf", type=int, default=10, help="instructions per frame")
    ap.add_argument("--frameskip", type=int, default=4)
    ap.add_argument("--score-reg", type=int, default=6)
    ap.add_argument("--variant", default="chip8", choices=["chip8", "schip"])
    a = ap.parse_args(argv)
    keys = (7, 9, 5, 8, 4, 6, 1, 2, 3, 10, 11, 12, 13, 14, 15, 0)[:a.actions]
    game = W.GameSpec(rom=open(a.rom, "rb").read(), instr_per_frame=a.ipf, frameskip=a.frameskip,
                      action_set=keys, score=(W.Term("reg", a.score_reg),), variant=a.variant)
    env = oracle.OracleEnv([game], a.envs, seed=a.seed)
    env.reset()
    acts = W.actions(a.action_seed, 0, a.steps, a.envs, a.actions + 1)
    _, r, d, h = env.rollout(acts, hashes=True)
    for s in range(a.steps):
        print(s, " ".join(f"{int(x):016x}" for x in h[s]))
    print("reward", f"{float(r.sum()):.0f}", "done", int(d.sum()))
    env.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
