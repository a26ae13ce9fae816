"""Bit-exact parity of the CUDA path (through the C-ABI) with the CPU oracle.

Small configurations are compared in full: every register, RAM byte, display
bit (via the per-step state hash and the canonical records), every
observation byte, reward and done flag. Full-size configurations run the
whole workload on the GPU in the launch configuration the benchmark uses and
compare a sample of instances, which the oracle steps one by one, at every
step.
"""
import numpy as np
import pytest

import oracle
from chip8_prog import prog
from paper_2510_01764_gb300 import workloads as W
from paper_2510_01764_gb300.workloads import Clause, GameSpec, Term

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


def hashes(env):
    return env.state_hash().cpu().numpy().view(np.uint64)


def full_compare(games, n, steps, *, seed=1, action_seed=1, game_of_env=None, quirks=0,
                 n_actions=None, launch=None, use_step_n=False, uid_of_env=None):
    """Step GPU and oracle side by side; compare everything at every step."""
    o = octax()
    env = o.Env(games, n, seed=seed, quirks=quirks, game_of_env=game_of_env, uid_of_env=uid_of_env)
    if launch:
        env.set_launch(**launch)
    ref = oracle.OracleEnv(games, n, seed=seed, quirks=quirks, game_of_env=game_of_env,
                           uid_of_env=uid_of_env)
    na = n_actions or games[0].n_actions
    acts = W.actions(action_seed, 0, steps, n, na + 1 if n_actions is None else n_actions)
    assert np.array_equal(env.reset().cpu().numpy(), ref.reset())
    assert np.array_equal(hashes(env), ref.hashes())
    a_dev = torch.from_numpy(acts).cuda()
    if use_step_n:
        obs, rew, done = env.step_n(a_dev)
        o2, r2, d2, _ = ref.rollout(acts, obs=True)
        assert np.array_equal(obs.cpu().numpy(), o2)
        assert np.array_equal(rew.cpu().numpy(), r2)
        assert np.array_equal(done.cpu().numpy(), d2)
        assert np.array_equal(hashes(env), ref.hashes())
    else:
        for s in range(steps):
            obs, rew, done = env.step(a_dev[s])
            o2, r2, d2 = ref.step(acts[s])
            assert np.array_equal(obs.cpu().numpy(), o2), f"obs step {s}"
            assert np.array_equal(rew.cpu().numpy(), r2), f"reward step {s}"
            assert np.array_equal(done.cpu().numpy(), d2), f"done step {s}"
            assert np.array_equal(hashes(env), ref.hashes()), f"state step {s}"
    g = env.get_state()
    r = ref.records()
    for f in oracle.RECORD_DTYPE.names:
        assert np.array_equal(g[f], r[f]), f
    return env, ref


# ----------------------------------------------------------------- small, full
def test_config_small_full_parity():
    """64 instances of the ~600 B template ROM, K = 10, frame skip 4, 1,000
    steps: every state, observation, reward and done flag."""
    w = W.cfg_small()
    full_compare(w.games, w.n_envs, w.n_steps, seed=w.seed, action_seed=w.action_seed,
                 n_actions=4)


def test_config_small_autotuned():
    """The small configuration (64 instances, 1,000 steps) in the shape the
    autotuner picks for 256-step calls (CTAs of fewer than 8 instances are
    candidates at this size), every instance compared at every step."""
    w = W.cfg_small()
    sampled_run(w, chunk=256, sample=np.arange(w.n_envs), autotune=True)


@pytest.mark.parametrize("launch", [
    dict(block=32, inst_per_warp=32, steps_per_launch=1, persistent=0, use_graph=0),
    dict(block=64, inst_per_warp=32, steps_per_launch=4, persistent=0, use_graph=1),
    dict(block=128, inst_per_warp=8, steps_per_launch=3, persistent=1, use_graph=1),
    dict(block=256, inst_per_warp=4, steps_per_launch=8, persistent=1, use_graph=0),
    dict(block=64, inst_per_warp=1, steps_per_launch=2, persistent=0, use_graph=1),
    dict(block=256, inst_per_warp=16, steps_per_launch=5, persistent=0, use_graph=1),
    dict(block=32, inst_per_warp=2, steps_per_launch=1, persistent=1, use_graph=0),
    dict(block=128, inst_per_warp=16, steps_per_launch=4, persistent=0, use_graph=1, writer_warps=2),
    dict(block=64, inst_per_warp=8, steps_per_launch=3, persistent=1, use_graph=1, writer_warps=2),
    dict(block=256, inst_per_warp=4, steps_per_launch=8, persistent=1, use_graph=0, writer_warps=4),
    dict(block=32, inst_per_warp=32, steps_per_launch=1, persistent=0, use_graph=1, writer_warps=1),
    dict(block=64, inst_per_warp=8, steps_per_launch=4, persistent=0, use_graph=1, balance=1),
    dict(block=256, inst_per_warp=7, steps_per_launch=4, persistent=0, use_graph=1, balance=1),
    dict(block=128, inst_per_warp=5, steps_per_launch=3, persistent=1, use_graph=1),
    dict(block=64, inst_per_warp=12, steps_per_launch=2, persistent=0, use_graph=0),
    dict(block=256, inst_per_warp=8, steps_per_launch=3, persistent=1, use_graph=0, balance=1),
    dict(block=128, inst_per_warp=16, steps_per_launch=2, persistent=0, use_graph=1, writer_warps=2,
         balance=1),
    dict(block=128, inst_per_warp=3, steps_per_launch=5, persistent=0, use_graph=1),
    dict(block=32, inst_per_warp=1, steps_per_launch=16, persistent=0, use_graph=1, balance=1),
    dict(block=256, inst_per_warp=2, steps_per_launch=64, persistent=1, use_graph=1),
])
def test_launch_configurations_agree(launch):
    w = W.cfg_small()
    full_compare(w.games, 200, 64, seed=3, action_seed=5, launch=launch, use_step_n=True)


def test_random_opcode_roms():
    """Random programs: every opcode, self-modifying code, stack faults, odd PCs."""
    games = [W.random_game(1000 + r) for r in range(32)]
    n = 256
    goe = (np.arange(n) % 32).astype(np.uint16)
    env, _ = full_compare(games, n, 150, seed=4, action_seed=4, game_of_env=goe)
    assert (env.get_state()["status"] & octax().STATUS_STACK_FAULT).any()


@pytest.mark.parametrize("quirks", [0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x3F])
def test_quirk_bits(quirks):
    games = [W.random_game(2000 + r) for r in range(8)]
    n = 96
    goe = (np.arange(n) % 8).astype(np.uint16)
    full_compare(games, n, 80, seed=9, action_seed=9, game_of_env=goe, quirks=quirks)


@pytest.mark.parametrize("n", [1, 31, 33, 100])
def test_ragged_instance_counts(n):
    w = W.cfg_small()
    full_compare(w.games, n, 40, seed=2, action_seed=2, launch=dict(block=64, inst_per_warp=32))


@pytest.mark.parametrize("launch", [None, dict(block=128, inst_per_warp=8, steps_per_launch=4,
                                                persistent=1, use_graph=1, writer_warps=1),
                                    dict(block=64, inst_per_warp=4, steps_per_launch=2,
                                         persistent=0, use_graph=1, balance=1)])
def test_mixed_games_timing_and_stacks(launch):
    """Different K and frame skip per game, stack_frames < frame skip,
    startup instructions that draw random numbers, shuffled instance order."""
    ts = [W.TemplateParams(seed=50 + i, size=300 + 100 * i, alu_ops=i, deco_pairs=i % 3,
                           wait_frames=i % 3) for i in range(4)]
    games = [
        W.replace(W.template_game(ts[0], instr_per_frame=5, frameskip=2), stack_frames=2),
        W.replace(W.template_game(ts[1], instr_per_frame=20, frameskip=3, score_limit=2),
                  stack_frames=2),
        W.replace(W.template_game(ts[2], instr_per_frame=7, frameskip=5, max_episode_steps=13),
                  stack_frames=2, startup_instrs=57),
        W.replace(W.random_game(77, frameskip=2), stack_frames=2, startup_instrs=33),
    ]
    n = 300
    goe = np.random.default_rng(0).integers(0, 4, n).astype(np.uint16)
    env, _ = full_compare(games, n, 120, seed=11, action_seed=12, game_of_env=goe, launch=launch,
                          use_step_n=launch is not None)
    env.sync()


@pytest.mark.parametrize("launch", [
    None,
    dict(block=64, inst_per_warp=16, steps_per_launch=4, persistent=1, use_graph=1),
    dict(block=128, inst_per_warp=8, steps_per_launch=3, persistent=0, use_graph=1, writer_warps=2),
])
def test_sticky_actions_and_noop_reset(launch):
    """§3.2 wrappers: sticky actions (p = 0.25) and no-op reset (0..30 no-op
    steps) on games with frequent episode ends, next to a game without
    either in the same launch; the previous action is compared in the state."""
    ts = [W.TemplateParams(seed=60 + i, size=400, wait_frames=i % 2) for i in range(3)]
    games = [
        W.replace(W.template_game(ts[0], score_limit=2, max_episode_steps=17), sticky_prob=0.25,
                  max_noops=30),
        W.replace(W.template_game(ts[1], max_episode_steps=9), max_noops=5, startup_instrs=23),
        W.template_game(ts[2], score_limit=3),
        W.replace(W.random_game(91), sticky_prob=0.9),
    ]
    n = 260
    goe = np.random.default_rng(3).integers(0, 4, n).astype(np.uint16)
    env, ref = full_compare(games, n, 90, seed=21, action_seed=22, game_of_env=goe, launch=launch,
                            use_step_n=launch is not None)
    la = env.get_state()["last_action"]
    assert (la == 4).any() and (la < 4).any()


def test_degenerate_games():
    """Edge cases of the descriptor: no actions (index 0 is the no-op), K = 1
    with one-frame observations, an episode limit of one step (a reset after
    every step), and 100,000 startup instructions drawing random numbers."""
    tp = W.TemplateParams(seed=21)
    games = [
        W.replace(W.template_game(tp), action_set=(), instr_per_frame=1, frameskip=1, stack_frames=1),
        W.replace(W.template_game(tp), instr_per_frame=3, frameskip=1, stack_frames=1, max_episode_steps=1),
        W.replace(W.random_game(44, frameskip=1), stack_frames=1, startup_instrs=100_000),
    ]
    n = 96
    goe = (np.arange(n) % 3).astype(np.uint16)
    env, _ = full_compare(games, n, 25, seed=8, action_seed=8, game_of_env=goe, n_actions=3)
    assert env.get_state()["episode_steps"][goe == 1].max() == 0


def test_reward_descriptor_memory_and_transforms():
    """Score from memory bytes written by FX33, several transforms, compound
    termination, truncation."""
    tp = W.TemplateParams(seed=5)
    g = W.template_game(tp)
    scratch = W.template_labels(tp)["scratch"]  # BCD buffer written by FX33
    g = W.replace(g, score=(Term("mem", scratch + 2, "raw"), Term("reg", 6, "dec_tens_minus_ones"),
                            Term("reg", 9, "zero_if_gt", 20), Term("reg", 8, "neg")),
                  term=(Clause(Term("reg", 6, "dec_ones"), "==", 3),
                        Clause(Term("mem", scratch + 1, "raw"), ">", 0),
                        Clause(Term("reg", 8, "nib_hi_minus_lo"), "<", -10)),
                  max_episode_steps=150)
    full_compare([g], 128, 200, seed=6, action_seed=6)
    full_compare([g], 128, 200, seed=6, action_seed=6, use_step_n=True,
                 launch=dict(block=64, inst_per_warp=16, steps_per_launch=5, persistent=0,
                             use_graph=1, writer_warps=4))


def test_out_of_range_actions():
    w = W.cfg_small()
    env, _ = full_compare(w.games, 64, 30, seed=1, action_seed=3, n_actions=7)
    assert (env.get_state()["status"] & octax().STATUS_BAD_ACTION).any()


def test_identity_independent_of_placement():
    """An instance's trajectory depends on (seed, uid, actions) only."""
    w = W.cfg_small()
    n = 96
    perm = np.random.default_rng(1).permutation(n).astype(np.uint32)
    full_compare(w.games, n, 50, seed=7, action_seed=7, uid_of_env=perm)


def test_reset_with_mask():
    o = octax()
    w = W.cfg_small()
    n = 80
    env = o.Env(w.games, n, seed=3)
    ref = oracle.OracleEnv(w.games, n, seed=3)
    env.reset()
    ref.reset()
    acts = W.actions(3, 0, 30, n)
    a_dev = torch.from_numpy(acts).cuda()
    for s in range(30):
        env.step(a_dev[s])
        ref.step(acts[s])
        if s in (10, 20):
            mask = (np.arange(n) % 3 == s % 2).astype(np.uint8)
            go = env.reset(mask=torch.from_numpy(mask).cuda(), out=torch.zeros((n, 4, 32, 64),
                                                                               dtype=torch.uint8,
                                                                               device="cuda"))
            ro = np.zeros((n, 4, 32, 64), dtype=np.uint8)
            ro_sel = ref.reset(mask)
            ro[mask == 1] = ro_sel[mask == 1]
            assert np.array_equal(go.cpu().numpy(), ro)
        assert np.array_equal(hashes(env), ref.hashes())


def test_checkpoint_roundtrip():
    """get_state / set_state: resuming from a checkpoint replays identically."""
    o = octax()
    games = [W.random_game(31), W.template_game(W.TemplateParams(seed=8))]
    n = 130
    goe = (np.arange(n) % 2).astype(np.uint16)
    env = o.Env(games, n, seed=5, game_of_env=goe)
    acts = torch.from_numpy(W.actions(8, 0, 60, n)).cuda()
    for s in range(30):
        env.step(acts[s])
    ck = env.get_state()
    h_ck = hashes(env)
    first = [tuple(t.cpu() for t in env.step(acts[s])) for s in range(30, 60)]
    env.set_state(ck)
    assert np.array_equal(hashes(env), h_ck)
    second = [tuple(t.cpu() for t in env.step(acts[s])) for s in range(30, 60)]
    for a, b in zip(first, second):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    # records restore into a fresh environment too (different launch config)
    env2 = o.Env(games, n, seed=5, game_of_env=goe)
    env2.set_launch(block=32, inst_per_warp=4)
    env2.set_state(ck)
    assert np.array_equal(hashes(env2), h_ck)


def test_memory_map_and_font_match_oracle():
    o = octax()
    g = GameSpec(rom=bytes(range(256)) * 14)
    env = o.Env([g], 2)
    ref = oracle.OracleEnv([g], 2)
    assert np.array_equal(env.get_state()["ram"], ref.records()["ram"])


def test_hand_programs_through_gpu():
    """The oracle's hand-assembled multiply program also runs on the GPU."""
    from test_oracle_pins import MUL8, RAMP
    g = prog(MUL8, instr_per_frame=20, frameskip=4)
    full_compare([g], 40, 8, seed=1)
    g = prog(RAMP, instr_per_frame=10, frameskip=4, score=(Term("reg", 6),),
             term=(Clause(Term("reg", 6), ">=", 20),))
    env, _ = full_compare([g], 40, 12, seed=1)


@pytest.mark.parametrize("variant", ["chip8", "schip"])
def test_code_as_data_through_gpu(variant):
    """A rewritten instruction (stale in the per-CTA micro-op table, so its
    page must be read as data) and an odd-address jump, on both variants and
    in two launch shapes: on CHIP-8, 128 threads x 8 instances per warp use
    the 16-byte micro-op table and 128 x 16 the 8-byte one (there the wide
    table would cost a resident CTA per SM); Super-CHIP always uses the
    8-byte table."""
    from test_oracle_pins import ODD, PATCH
    for launch in (dict(block=128, inst_per_warp=8, steps_per_launch=4, persistent=0, use_graph=1),
                   dict(block=128, inst_per_warp=16, steps_per_launch=2, persistent=1, use_graph=0)):
        g1 = prog(PATCH, instr_per_frame=3, frameskip=4, variant=variant)
        g2 = GameSpec(rom=ODD, instr_per_frame=3, frameskip=4, action_set=(7, 9, 5, 8), variant=variant)
        env, ref = full_compare([g1, g2], 64, 4, seed=2, launch=launch,
                                game_of_env=(np.arange(64) % 2).astype(np.uint16))
        V = env.get_state()["V"]
        assert (V[0::2, 10] == 9).all() and (V[1::2, 12] == 7).all()


from test_oracle_pins import SPRITE_PAGE_DATA, SPRITE_PAGE_WORDS  # noqa: E402

EDGE_PROGRAMS = [
    # FX33 across the end of memory into page 0, FX65 back, then a sprite read
    # from the written (dirty) page 0
    [0x6A7B, 0xAFFE, 0xFA33, 0xAFFE, 0xF265, 0xA000, 0x6305, 0x6404, 0xD345, 0x1212],
    # FX55 into the last page, then a sprite whose rows wrap from 0xFFF to
    # 0x000, clipped at the right and bottom edges, then drawn at wrapped
    # coordinates and erased (VF = 1)
    [0x60FF, 0x6181, 0x623C, 0xAFFD, 0xF255, 0xAFFD, 0x603C, 0x611E, 0xD015,
     0x6045, 0x6123, 0xD015, 0xD015, 0x121A],
    # unbounded recursion: the 17th call overflows (STACK_FAULT, wraps), again and again
    [0x2204, 0x1202, 0x7001, 0x2204],
    # return on an empty stack, then execution from low memory
    [0x6001, 0x00EE, 0x1204],
    # undefined encodings and an ignored 0NNN
    [0x8018, 0x801F, 0x5011, 0x9012, 0xE000, 0xE19F, 0xF0FF, 0xF001, 0x0123, 0x1212],
    # BNNN past the end of memory (wraps to 0x0FE) and through low memory
    [0x60FF, 0xBFFF],
    # FX0A: wait for the step's key, count the presses
    [0xF00A, 0x7101, 0x1200],
    # sprites on a written page: one outside the written bytes, one rewritten
    # by FX55, one inside the written address range but unchanged
    (SPRITE_PAGE_WORDS, SPRITE_PAGE_DATA),
]


@pytest.mark.parametrize("variant,quirks", [("chip8", 0), ("chip8", 0x3F), ("schip", 0)])
def test_edge_programs_through_gpu(variant, quirks):
    """Memory wrap for FX33/FX55/FX65 and sprite rows, reads from written
    pages, stack overflow and underflow, undefined opcodes, BNNN past 0xFFF,
    FX0A with the step's key: whole-state parity at every step, seven
    programs interleaved in one environment."""
    games = [prog(*(p if isinstance(p, tuple) else (p,)), instr_per_frame=10, frameskip=4, variant=variant)
             for p in EDGE_PROGRAMS]
    n = 4 * len(games)
    goe = (np.arange(n) % len(games)).astype(np.uint16)
    env, ref = full_compare(games, n, 12, seed=3, action_seed=3, game_of_env=goe, quirks=quirks)
    st = ref.records()["status"]
    assert (st[2::len(games)] & oracle.ST_STACK_FAULT).all()
    assert (st[3::len(games)] & oracle.ST_STACK_FAULT).all()
    assert (st[4::len(games)] & oracle.ST_BAD_OP).all()


def test_autotune_leaves_no_trace():
    o = octax()
    w = W.cfg_small()
    n = 256
    env = o.Env(w.games, n, seed=1)
    acts = torch.from_numpy(W.actions(1, 0, 40, n)).cuda()
    env.step_n(acts[:20])
    h0 = hashes(env)
    ms = env.autotune(8)
    assert ms > 0
    assert np.array_equal(hashes(env), h0)
    o1 = env.step_n(acts[20:])
    ref = o.Env(w.games, n, seed=1)
    ref.set_launch(block=32, inst_per_warp=32, steps_per_launch=1, persistent=0, use_graph=0)
    ref.step_n(acts[:20])
    o2 = ref.step_n(acts[20:])
    for x, y in zip(o1, o2):
        assert torch.equal(x, y)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_step_matches_device_step(pinned):
    """Pinned buffers are written by the kernel directly; pageable ones are staged."""
    o = octax()
    w = W.cfg_small()
    n = 128
    a = W.actions(1, 0, 10, n)
    e1 = o.Env(w.games, n, seed=1)
    e2 = o.Env(w.games, n, seed=1)
    out = (torch.empty((n, 4, 32, 64), dtype=torch.uint8, pin_memory=pinned),
           torch.empty(n, dtype=torch.float32, pin_memory=pinned),
           torch.empty(n, dtype=torch.uint8, pin_memory=pinned))
    for s in range(10):
        d = e1.step(torch.from_numpy(a[s]).cuda())
        act = torch.from_numpy(a[s].copy())
        h = e2.step_host(act.pin_memory() if pinned else act, out=out)
        for x, y in zip(d, h):
            assert torch.equal(x.cpu(), y)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("variant", ["chip8", "schip"])
def test_packed_host_step_matches_oracle(pinned, variant):
    """step_host_packed (mapped pinned buffers, or staged pageable ones, the
    staging shared with step_host) against the oracle's packed frames."""
    o = octax()
    g = W.replace(W.template_game(W.TemplateParams(seed=3), score_limit=2, max_episode_steps=9),
                  variant=variant)
    n = 70
    env = o.Env([g], n, seed=4)
    ref = oracle.OracleEnv([g], n, seed=4)
    env.reset()
    ref.reset()
    acts = W.actions(4, 0, 24, n, 5)
    W_ = 32 if variant == "chip8" else 128
    out = (torch.empty((n, 4, W_), dtype=torch.int64, pin_memory=pinned),
           torch.empty(n, dtype=torch.float32, pin_memory=pinned),
           torch.empty(n, dtype=torch.uint8, pin_memory=pinned))
    for s in range(24):
        o2, r2, d2 = ref.step(acts[s])
        act = torch.from_numpy(acts[s].copy())
        if s % 3 == 2:
            obs, rew, done = env.step_host(act)
            assert np.array_equal(obs.numpy(), o2)
        else:
            obs, rew, done = env.step_host_packed(act.pin_memory() if pinned else act, out=out)
            assert np.array_equal(obs.numpy().view(np.uint64), pack_frames(o2))
        assert np.array_equal(rew.numpy(), r2) and np.array_equal(done.numpy(), d2)
    assert np.array_equal(hashes(env), ref.hashes())


def test_sync_timeout_is_reported():
    """octax_sync returns ETIMEOUT (not a hang) while work is still running."""
    o = octax()
    w = W.cfg_divergence(n_envs=16384, n_steps=48)
    env = o.Env(w.games, w.n_envs, seed=1, game_of_env=w.game_of_env)
    acts = torch.zeros((48, w.n_envs), dtype=torch.uint8, device="cuda")
    out = env.step_n(acts)
    with pytest.raises(o.OctaxError) as ei:
        env.sync(timeout_ms=0)
    assert ei.value.code in (o.ETIMEOUT,)
    env.sync(timeout_ms=-1)
    del out


# ----------------------------------------------------------------- full size, sampled
def sampled_run(w, *, chunk, sample, launch=None, use_step_n=True, autotune=False):
    """Run the whole workload on the GPU; compare `sample` rows with the
    oracle at every step (obs, reward, done) and the state hash at every
    chunk boundary. With autotune, the launch shape is the one octax_autotune
    picks for chunk-step calls on the first chunk of actions, as the
    benchmark does before it times the same workload in chunk-step calls."""
    o = octax()
    env = o.Env(w.games, w.n_envs, seed=w.seed, quirks=w.quirks, game_of_env=w.game_of_env)
    if launch:
        env.set_launch(**launch)
    if autotune:
        a0 = torch.from_numpy(W.actions(w.action_seed, 0, chunk, w.n_envs, w.games[0].n_actions)).cuda()
        env.autotune(chunk, a0)
        print(f"{w.name}: autotuned launch for {chunk}-step calls: {env.launch}")
        del a0
    goe = None if w.game_of_env is None else w.game_of_env[sample]
    ref = oracle.OracleEnv(w.games, len(sample), seed=w.seed, quirks=w.quirks, game_of_env=goe,
                           uid_of_env=sample.astype(np.uint32))
    idx = torch.from_numpy(sample.astype(np.int64)).cuda()
    assert np.array_equal(env.reset()[idx].cpu().numpy(), ref.reset())
    n_actions = w.games[0].n_actions
    T = chunk
    obs_buf = torch.empty((T, w.n_envs, 4) + env.frame, dtype=torch.uint8, device="cuda")
    rew_buf = torch.empty((T, w.n_envs), dtype=torch.float32, device="cuda")
    done_buf = torch.empty((T, w.n_envs), dtype=torch.uint8, device="cuda")
    n_done = 0
    for lo in range(0, w.n_steps, T):
        hi = min(lo + T, w.n_steps)
        acts = W.actions(w.action_seed, lo, hi, w.n_envs, n_actions)
        a_dev = torch.from_numpy(acts).cuda()
        c = hi - lo
        out = (obs_buf[:c], rew_buf[:c], done_buf[:c])
        if use_step_n:
            env.step_n(a_dev, out=out)
        else:
            for s in range(c):
                env.step(a_dev[s], out=(obs_buf[s], rew_buf[s], done_buf[s]))
        o2, r2, d2, h2 = ref.rollout(acts[:, sample], obs=True, hashes=True)
        assert np.array_equal(obs_buf[:c][:, idx].cpu().numpy(), o2), f"obs in steps {lo}..{hi}"
        assert np.array_equal(rew_buf[:c][:, idx].cpu().numpy(), r2), f"reward in {lo}..{hi}"
        assert np.array_equal(done_buf[:c][:, idx].cpu().numpy(), d2), f"done in {lo}..{hi}"
        gh = env.state_hash()[idx].cpu().numpy().view(np.uint64)
        assert np.array_equal(gh, h2[-1]), f"state after step {hi}"
        n_done += int(done_buf[:c].sum().item())
    return env, n_done


def pick(n, k, seed=0, extra=()):
    rng = np.random.default_rng(seed)
    s = set(int(v) for v in rng.choice(n, size=k, replace=False))
    s.update(e for e in extra if 0 <= e < n)
    return np.array(sorted(s), dtype=np.int64)


def test_config_scale_sampled():
    """16,384 template instances x 20,000 steps with auto-reset (score >= 20
    or 5,000 steps), plain one-launch-per-step kernel."""
    w = W.cfg_scale()
    sample = pick(w.n_envs, 24, 1, extra=(0, 31, 32, 63, 64, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=50, sample=sample, use_step_n=False)
    assert n_done > 0


def test_config_scale_sampled_persistent_graph():
    """Same workload through octax_step_n (CUDA graph, 4 steps per launch)."""
    w = W.cfg_scale(n_steps=6000)
    sample = pick(w.n_envs, 16, 2, extra=(5, w.n_envs - 2))
    sampled_run(w, chunk=40, sample=sample,
                launch=dict(block=128, inst_per_warp=8, steps_per_launch=4, persistent=1,
                            use_graph=1))


def test_config_scale_sampled_writer_warps():
    """The full 20,000-step workload through the warp-specialised kernel."""
    w = W.cfg_scale()
    sample = pick(w.n_envs, 16, 5, extra=(7, w.n_envs - 3))
    env, n_done = sampled_run(w, chunk=64, sample=sample,
                              launch=dict(block=256, inst_per_warp=16, steps_per_launch=8,
                                          persistent=0, use_graph=1, writer_warps=4))
    env.sync()
    assert n_done > 0


def test_config_scale_sampled_balanced():
    """The full workload in the launch configuration the benchmark times:
    256 threads x 7 instances per warp, balanced waves, 32 steps per
    graph-replayed launch."""
    w = W.cfg_scale()
    sample = pick(w.n_envs, 16, 6, extra=(53, 54, 107, 108, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=64, sample=sample,
                              launch=dict(block=256, inst_per_warp=7, steps_per_launch=32,
                                          persistent=0, use_graph=1, balance=1))
    assert n_done > 0


def test_config_wrappers_sampled():
    """The template workload behind sticky actions (p = 0.25) and no-op resets
    (0-30 steps), 16,384 instances x 3,000 steps in the benchmark's launch
    shape (the wrapper kernel variant); episodes truncated at 700 steps here
    so that every instance goes through auto-resets with no-op steps."""
    w = W.cfg_wrappers(n_steps=3000)
    w.games = [W.replace(w.games[0], max_episode_steps=700)]
    sample = pick(w.n_envs, 16, 12, extra=(0, 53, 54, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=64, sample=sample,
                              launch=dict(block=256, inst_per_warp=7, steps_per_launch=32,
                                          persistent=0, use_graph=1, balance=1))
    assert n_done > 0


@pytest.mark.parametrize("spl", [64, 128, 256])
def test_config_wrappers_long_launches(spl):
    """The wrappers workload (episodes truncated at 700 steps, so every
    instance resets through its no-op steps) in launches of 64, 128 and 256
    steps inside 256-step calls, the benchmark's default call length for
    16,384 instances; 3,000 steps, so the last call and its launches are
    ragged."""
    w = W.cfg_wrappers(n_steps=3000)
    w.games = [W.replace(w.games[0], max_episode_steps=700)]
    sample = pick(w.n_envs, 12, 40 + spl, extra=(0, 55, 56, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=256, sample=sample,
                              launch=dict(block=256, inst_per_warp=7, steps_per_launch=spl,
                                          persistent=0, use_graph=1, balance=1))
    assert n_done > 0


@pytest.mark.parametrize("config", ["wrappers", "scale"])
def test_config_autotuned_256(config):
    """The 16,384-instance workloads (the full 20,000-step scale workload;
    the wrappers one with episodes truncated at 700 steps) in the shape the
    autotuner picks for 256-step calls, whose candidates now include
    launches of up to 256 steps."""
    if config == "wrappers":
        w = W.cfg_wrappers(n_steps=3000)
        w.games = [W.replace(w.games[0], max_episode_steps=700)]
    else:
        w = W.cfg_scale()
    sample = pick(w.n_envs, 16, 50 + len(config), extra=(1, 111, 112, w.n_envs - 1))
    env, n_done = sampled_run(w, chunk=256, sample=sample, autotune=True)
    assert n_done > 0


@pytest.mark.parametrize("balance", [0, 1])
def test_config_batch_sampled(balance):
    """65,536 instances over 16 ROMs (K from {5,8,10,15,20}, uneven episodes),
    16 frames per persistent graph-captured launch."""
    w = W.cfg_batch()
    goe = w.game_of_env
    per_game = [np.nonzero(goe == g)[0][:2] for g in range(16)]
    sample = np.unique(np.concatenate(per_game + [pick(w.n_envs, 16, 3)]))
    sampled_run(w, chunk=32, sample=sample,
                launch=dict(block=64, inst_per_warp=16, steps_per_launch=4, persistent=1,
                            use_graph=1, balance=balance))


@pytest.mark.parametrize("T", [20, 32])
def test_config_divergence_autotuned(T):
    """262,144 random-opcode instances x 2,000 steps in the launch shape the
    autotuner picks for T-step calls (T = 32: the benchmark's default; T =
    20: a 20-step benchmark run), stepped in T-step calls like the
    benchmark's timed region."""
    w = W.cfg_divergence()
    sample = pick(w.n_envs, 24, 14, extra=(0, 1, 63, 64, w.n_envs - 1))
    sampled_run(w, chunk=T, sample=sample, autotune=True)


@pytest.mark.parametrize("spl,persistent,chunk", [(16, 0, 32), (16, 1, 32), (32, 0, 32), (32, 1, 32),
                                                  (20, 0, 20), (20, 1, 20)])
def test_config_divergence_bench_shapes(spl, persistent, chunk):
    """The divergence workload in the shapes the autotuner picks for it
    (128 threads x 16 instances per warp, graph replay) at 16, 20 and 32
    steps per launch, with and without the persistent queue, stepped in
    calls of the benchmark's length."""
    w = W.cfg_divergence()
    sample = pick(w.n_envs, 12, 15 + spl + persistent, extra=(2, 127, w.n_envs - 2))
    sampled_run(w, chunk=chunk, sample=sample,
                launch=dict(block=128, inst_per_warp=16, steps_per_launch=spl, persistent=persistent,
                            use_graph=1))


@pytest.mark.parametrize("T", [20, 32, 64])
def test_config_batch_autotuned(T):
    """65,536 instances over 16 ROMs in the autotuned shape for T-step calls
    (64: the benchmark's default call length for this workload)."""
    w = W.cfg_batch()
    goe = w.game_of_env
    per_game = [np.nonzero(goe == g)[0][:1] for g in range(16)]
    sample = np.unique(np.concatenate(per_game + [pick(w.n_envs, 8, 16)]))
    sampled_run(w, chunk=T, sample=sample, autotune=True)


@pytest.mark.parametrize("block,spl,chunk", [(128, 32, 32), (256, 32, 32), (256, 20, 20)])
def test_config_batch_bench_shape(block, spl, chunk):
    """The batch workload in the shapes the autotuner picked for it: 128 or
    256 threads x 16 instances per warp, 20 or 32 steps per graph-replayed
    launch."""
    w = W.cfg_batch()
    goe = w.game_of_env
    per_game = [np.nonzero(goe == g)[0][-1:] for g in range(16)]
    sample = np.unique(np.concatenate(per_game + [pick(w.n_envs, 8, 17 + block)]))
    sampled_run(w, chunk=chunk, sample=sample,
                launch=dict(block=block, inst_per_warp=16, steps_per_launch=spl, persistent=0, use_graph=1))


def test_config_divergence_sampled():
    """262,144 instances of random-opcode ROMs x 2,000 steps."""
    w = W.cfg_divergence()
    sample = pick(w.n_envs, 32, 4, extra=(0, 1, w.n_envs - 1))
    sampled_run(w, chunk=8, sample=sample,
                launch=dict(block=128, inst_per_warp=32, steps_per_launch=4, persistent=0,
                            use_graph=1))


def test_four_million_instances_sampled():
    """4,194,339 instances (2^22 + 35: past every 32-bit byte offset of the
    observation and state arrays, a ragged last group), 3 steps with
    truncation after 2 (every instance auto-resets at once), in the
    benchmark's launch shape; packed observations keep the output at 4.3 GB
    per step. Sampled instances at both ends and around 2^21 and 2^22."""
    o = octax()
    g = W.template_game(W.TemplateParams(seed=2), max_episode_steps=2)
    n = (1 << 22) + 35
    sample = pick(n, 12, 11, extra=(0, 1, (1 << 21) - 1, 1 << 21, (1 << 22) - 1, 1 << 22, n - 2, n - 1))
    env = o.Env([g], n, seed=3)
    env.set_launch(block=256, inst_per_warp=7, steps_per_launch=32, persistent=0, use_graph=1, balance=1)
    ref = oracle.OracleEnv([g], len(sample), seed=3, uid_of_env=sample.astype(np.uint32))
    idx = torch.from_numpy(sample).cuda()
    steps = 3                      # both sides start from the reset octax_create / the oracle ran
    acts = W.actions(9, 0, steps, n, 4)
    a_dev = torch.from_numpy(acts).cuda()
    obs, rew, done = env.step_n_packed(a_dev)
    o2, r2, d2, h2 = ref.rollout(acts[:, sample], obs=True, hashes=True)
    assert np.array_equal(obs[:, idx].cpu().numpy().view(np.uint64), pack_frames(o2))
    assert np.array_equal(rew[:, idx].cpu().numpy(), r2)
    assert np.array_equal(done[:, idx].cpu().numpy(), d2)
    assert int(done[1].sum().item()) == n and int(done[0].sum().item()) == 0
    assert np.array_equal(env.state_hash()[idx].cpu().numpy().view(np.uint64), h2[-1])
    del obs, rew, done, env
    torch.cuda.empty_cache()


# ----------------------------------------------------------------- packed observations
def pack_frames(obs_u8: np.ndarray) -> np.ndarray:
    """uint8 0/1 frames [..., H, W] -> u64 words [..., H * W / 64] (bit x of a
    word = pixel x of its 64-pixel run), the layout octax_step_n_packed writes."""
    b = np.packbits(obs_u8, axis=-1, bitorder="little")
    return b.view("<u8").reshape(obs_u8.shape[:-2] + (-1,))


@pytest.mark.parametrize("launch", [
    None,
    dict(block=256, inst_per_warp=7, steps_per_launch=8, persistent=0, use_graph=1, balance=1),
    dict(block=64, inst_per_warp=16, steps_per_launch=3, persistent=1, use_graph=1),
    dict(block=128, inst_per_warp=16, steps_per_launch=4, persistent=0, use_graph=1, writer_warps=2),
])
def test_packed_observations(launch):
    """step_n_packed: the packed frames are the uint8 frames bit for bit, and
    rewards, done flags (auto-resets included) and state match the oracle;
    packed and uint8 calls interleave on one environment."""
    o = octax()
    games = [W.template_game(W.TemplateParams(seed=4), score_limit=3, max_episode_steps=37),
             W.random_game(55)]
    n = 150
    goe = (np.arange(n) % 2).astype(np.uint16)
    env = o.Env(games, n, seed=6, game_of_env=goe)
    if launch:
        env.set_launch(**launch)
    ref = oracle.OracleEnv(games, n, seed=6, game_of_env=goe)
    env.reset()
    ref.reset()
    acts = W.actions(6, 0, 60, n, 5)
    a_dev = torch.from_numpy(acts).cuda()
    for lo, hi, packed in ((0, 20, True), (20, 30, False), (30, 60, True)):
        o2, r2, d2, _ = ref.rollout(acts[lo:hi], obs=True)
        if packed:
            obs, rew, done = env.step_n_packed(a_dev[lo:hi])
            assert np.array_equal(obs.cpu().numpy().view(np.uint64), pack_frames(o2))
        else:
            obs, rew, done = env.step_n(a_dev[lo:hi])
            assert np.array_equal(obs.cpu().numpy(), o2)
        assert np.array_equal(rew.cpu().numpy(), r2)
        assert np.array_equal(done.cpu().numpy(), d2)
        assert np.array_equal(hashes(env), ref.hashes())
    assert int(done.sum()) >= 0
