"""Bit-exact parity of the Super-CHIP variant (the 128x64 extension §5 names)
between the CUDA path and the CPU oracle: states, [S][64][128] observations,
rewards and done flags at every step, over the hires template game, random
programs that mix lores and hires, every launch shape family, the wrappers,
quirk bits, checkpoints and the serving path.
"""
import numpy as np
import pytest

import oracle
from chip8_prog import prog
from paper_2510_01764_gb300 import workloads as W
from test_gpu_parity import full_compare, hashes, pick, sampled_run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_01764_gb300 import build

    build.build()
    oracle.build()


def octax():
    from paper_2510_01764_gb300 import octax as o

    return o


def template(seed=3, **kw):
    return W.schip_template_game(W.TemplateParams(seed=seed, size=700, deco_pairs=1), **kw)


def test_schip_template_full_parity():
    """64 hires template instances, 300 steps, auto-reset on score >= 6."""
    env, ref = full_compare([template(score_limit=6)], 64, 300, seed=3, action_seed=3)
    assert env.get_state()["hires"].mean() > 0.8  # just-reset instances are in lores until 00FF


@pytest.mark.parametrize("launch", [
    dict(block=32, inst_per_warp=32, steps_per_launch=1, persistent=0, use_graph=0),
    dict(block=64, inst_per_warp=8, steps_per_launch=4, persistent=0, use_graph=1, balance=1),
    dict(block=128, inst_per_warp=7, steps_per_launch=3, persistent=1, use_graph=1),
    dict(block=256, inst_per_warp=4, steps_per_launch=8, persistent=0, use_graph=1),
    dict(block=64, inst_per_warp=1, steps_per_launch=6, persistent=0, use_graph=1),
    dict(block=128, inst_per_warp=2, steps_per_launch=60, persistent=1, use_graph=1, balance=1),
    dict(block=32, inst_per_warp=3, steps_per_launch=4, persistent=0, use_graph=0),
])
def test_schip_launch_configurations(launch):
    full_compare([template(score_limit=4, max_episode_steps=50)], 150, 60, seed=5, action_seed=5,
                 launch=launch, use_step_n=True)


def test_random_schip_programs_both_modes():
    """Random programs over all CHIP-8 and SCHIP forms: scrolls, mode
    switches, 16x16 sprites, big glyphs, flag registers, stack faults."""
    games = [W.random_schip_game(3000 + r) for r in range(32)]
    n = 256
    goe = (np.arange(n) % 32).astype(np.uint16)
    env, _ = full_compare(games, n, 120, seed=4, action_seed=4, game_of_env=goe)
    st = env.get_state()
    assert (st["hires"] == 1).any() and (st["hires"] == 0).any()


@pytest.mark.parametrize("quirks", [0x10, 0x3F])
def test_schip_quirks(quirks):
    games = [W.random_schip_game(4000 + r) for r in range(8)] + [template(seed=9)]
    n = 90
    goe = (np.arange(n) % 9).astype(np.uint16)
    full_compare(games, n, 80, seed=9, action_seed=9, game_of_env=goe, quirks=quirks)


def test_schip_hand_programs():
    """Exit (00FD), lores 16x16 sprites, scroll down in both modes."""
    big = bytes(range(1, 33))
    g = prog([0x00FE, 0x6010, 0x6108, 0xA220, 0xD010, 0x00C3, 0x00FF, 0x00C2, 0xD010, 0x00FB,
              0x00FD, 0x1200, 0, 0, 0, 0], data=big, variant="schip", instr_per_frame=4)
    env, _ = full_compare([g], 33, 6, seed=1)
    assert (env.get_state()["status"] & octax().STATUS_EXIT).all()


def test_schip_wrappers_and_mixed_timing():
    games = [W.replace(template(seed=11, score_limit=3, max_episode_steps=30), sticky_prob=0.25,
                       max_noops=7, stack_frames=2),
             W.replace(W.random_schip_game(77, frameskip=2, instr_per_frame=7), stack_frames=2,
                       startup_instrs=31),
             W.replace(template(seed=12), frameskip=2, stack_frames=2)]
    n = 120
    goe = np.random.default_rng(2).integers(0, 3, n).astype(np.uint16)
    full_compare(games, n, 70, seed=13, action_seed=13, game_of_env=goe,
                 launch=dict(block=64, inst_per_warp=8, steps_per_launch=4, persistent=1, use_graph=1),
                 use_step_n=True)


def test_schip_checkpoint_roundtrip():
    o = octax()
    games = [W.random_schip_game(31), template(seed=8)]
    n = 70
    goe = (np.arange(n) % 2).astype(np.uint16)
    env = o.Env(games, n, seed=5, game_of_env=goe)
    acts = torch.from_numpy(W.actions(8, 0, 40, n)).cuda()
    for s in range(20):
        env.step(acts[s])
    ck = env.get_state()
    h_ck = hashes(env)
    first = [tuple(t.cpu() for t in env.step(acts[s])) for s in range(20, 40)]
    env2 = o.Env(games, n, seed=5, game_of_env=goe)
    env2.set_state(ck)
    assert np.array_equal(hashes(env2), h_ck)
    second = [tuple(t.cpu() for t in env2.step(acts[s])) for s in range(20, 40)]
    for a, b in zip(first, second):
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def test_schip_rejections():
    o = octax()
    with pytest.raises(o.OctaxError):
        o.Env([W.template_game(W.TemplateParams(seed=1)), template()], 4,
              game_of_env=np.array([0, 1, 0, 1], np.uint16))
    env = o.Env([template()], 8)
    with pytest.raises(o.OctaxError):
        env.set_launch(block=128, inst_per_warp=8, writer_warps=1)
    with pytest.raises(o.OctaxError):
        env.set_launch(block=256, inst_per_warp=32)   # 256 x 1 KB displays exceed shared memory


def test_schip_server_requests_match_oracle():
    o = octax()
    gs = [template(seed=s, score_limit=3) for s in (1, 2)] + [W.random_schip_game(5)]
    srv = o.Server(gs, memory_budget_bytes=2000 * 6000)
    rng = np.random.default_rng(4)
    reqs = [dict(game=int(rng.integers(0, 3)), actions=rng.integers(0, 5, size=(5, int(n)), dtype=np.uint8),
                 seed=int(rng.integers(0, 2 ** 62))) for n in (1, 17, 64, 200)]
    ids = [srv.submit(r["game"], r["actions"], r["seed"]) for r in reqs]
    for i in ids:
        srv.wait(i, timeout_ms=60000)
    outs = [tuple(t.cpu() for t in srv.outputs(i)) for i in ids]
    srv.close()
    for r, got in zip(reqs, outs):
        n = r["actions"].shape[1]
        ref = oracle.OracleEnv(gs, n, seed=r["seed"], game_of_env=np.full(n, r["game"], np.uint16))
        ref.reset()
        ob, rw, dn, _ = ref.rollout(r["actions"], obs=True)
        assert np.array_equal(got[0].numpy(), ob)
        assert np.array_equal(got[1].numpy(), rw)
        assert np.array_equal(got[2].numpy(), dn)


def test_schip_scale_sampled():
    """16,384 hires template instances x 4,000 steps (K = 20), balanced
    graph-replayed launches; sampled instances against the oracle."""
    w = W.cfg_schip()
    sample = pick(w.n_envs, 12, 7, extra=(0, 53, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=50, sample=sample,
                              launch=dict(block=128, inst_per_warp=7, steps_per_launch=8, persistent=0,
                                          use_graph=1, balance=1))
    assert n_done > 0


def test_schip_packed_observations():
    from test_gpu_parity import pack_frames
    o = octax()
    games = [template(seed=5, score_limit=3, max_episode_steps=25), W.random_schip_game(61)]
    n = 90
    goe = (np.arange(n) % 2).astype(np.uint16)
    env = o.Env(games, n, seed=2, game_of_env=goe)
    ref = oracle.OracleEnv(games, n, seed=2, game_of_env=goe)
    env.reset()
    ref.reset()
    acts = W.actions(2, 0, 40, n, 5)
    obs, rew, done = env.step_n_packed(torch.from_numpy(acts).cuda())
    o2, r2, d2, _ = ref.rollout(acts, obs=True)
    assert obs.shape == (40, n, 4, 128)
    assert np.array_equal(obs.cpu().numpy().view(np.uint64), pack_frames(o2))
    assert np.array_equal(rew.cpu().numpy(), r2) and np.array_equal(done.cpu().numpy(), d2)
    assert np.array_equal(hashes(env), ref.hashes())


def test_schip_scale_autotuned_64():
    """The 16,384-instance hires workload (4,000 steps) in the shape the
    autotuner picks for the benchmark's default 64-step calls."""
    w = W.cfg_schip()
    sample = pick(w.n_envs, 10, 27, extra=(1, 111, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=64, sample=sample, autotune=True)
    assert n_done > 0
