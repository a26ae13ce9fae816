"""The §4.1 actor-critic network on the tensor cores, against the float64
oracle (oracle/policy.py), through the C-ABI.

Tolerances (floating point; the environment step itself stays bit-exact):
- against the oracle with bfloat16 storage (weights and stored activations
  rounded as the kernels store them, products summed in float64): the
  kernels differ by fp32 accumulation order, and where that order decides
  the bfloat16 rounding of a stored activation the two sides differ by one
  bfloat16 ulp of it (2^-8 relative, up to 0.016 for activations near 4),
  damped by the layers after it; measured worst case 1.3e-3 over ~10^4
  evaluations, typical 1e-4. Bound: |logit or value difference| <= 5e-3 *
  max(1, RMS of the oracle's logits);
- against the float64 oracle: bfloat16 weights and activations (unit
  roundoff 2^-9) through five layers, |difference| <= 5e-2 * max(1, RMS);
- sampled actions: the kernel's draw from its own fp32 logits equals the
  float64 inverse-CDF draw with the same uniform number wherever that number
  lies more than 1e-5 from a CDF boundary.
"""
import numpy as np
import pytest

import oracle
from oracle import policy as P
from paper_2510_01764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_BF16, TOL_F64, MARGIN = 5e-3, 5e-2, 1e-5


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


def pack(obs_u8: np.ndarray) -> np.ndarray:
    """uint8 frames [..., 32, 64] -> int64 words [..., 32] (bit x = pixel x)."""
    b = np.packbits(obs_u8, axis=-1, bitorder="little")
    return b.view("<u8").reshape(obs_u8.shape[:-1]).view(np.int64)


def random_frames(n, density, seed):
    rng = np.random.default_rng(seed)
    return (rng.random((n, 4, 32, 64)) < density).astype(np.uint8)


def env_frames(n, steps, seed):
    """Observation stacks of template games played with random actions (oracle)."""
    g = W.template_game(W.TemplateParams(seed=seed))
    ref = oracle.OracleEnv([g], n, seed=seed)
    ref.reset()
    acts = W.actions(seed, 0, steps, n, g.n_actions + 1)
    o, _, _, _ = ref.rollout(acts, obs=True)
    return o[-1]


def philox_u(seed, step, n, idx=None):
    """The kernel's uniform numbers from the oracle's own Philox4x32-10:
    key = seed (low word first), counter = (instance, step, 0, 0), word 0
    (for instances 0..n-1, or those in idx)."""
    k = (seed & 0xFFFFFFFF, seed >> 32)
    inst = range(n) if idx is None else (int(i) for i in idx)
    words = np.array([oracle.philox4x32_10((i, step, 0, 0), k)[0] for i in inst], dtype=np.uint64)
    return P.uniform_from_word(words)


def check_outputs(params, obs, lg, v):
    l16, v16 = P.forward(params, obs, storage="bf16")
    l64, v64 = P.forward(params, obs)
    scale = max(1.0, float(np.sqrt((l64 ** 2).mean())))
    lg, v = lg.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    e16 = max(np.abs(lg - l16).max(), np.abs(v - v16).max())
    e64 = max(np.abs(lg - l64).max(), np.abs(v - v64).max())
    print(f"n={len(obs)}: max |gpu - oracle(bf16)| = {e16:.3g}, max |gpu - oracle(f64)| = {e64:.3g}, "
          f"logit rms {scale:.3g}")
    assert e16 <= TOL_BF16 * scale, e16
    assert e64 <= TOL_F64 * scale, e64
    return l16


@pytest.mark.parametrize("n,density,L", [(1, 0.1, 5), (8, 0.3, 5), (129, 0.05, 17), (300, 0.15, 6)])
def test_forward_matches_oracle(n, density, L):
    """Ragged batches of 8 and tiles of 128, packed and uint8 inputs."""
    o = octax()
    params = W.policy_params(10 + n, L)
    obs = random_frames(n, density, n)
    pol = o.Policy(params, max_envs=max(n, 64))
    words = torch.from_numpy(pack(obs)).cuda()
    lg, v, a = pol.forward(words, seed=5, step=3)
    lg2, v2, a2 = pol.forward_u8(torch.from_numpy(obs).cuda(), seed=5, step=3)
    pol.sync()
    assert torch.equal(lg, lg2) and torch.equal(v, v2) and torch.equal(a, a2)
    check_outputs(params, obs, lg, v)


def test_forward_on_game_frames_and_sampling():
    o = octax()
    n, L = 256, 5
    params = W.policy_params(3, L)
    obs = env_frames(n, 30, 2)
    pol = o.Policy(params, max_envs=n)
    seed, step = 0x1234_5678_9ABC, 7
    lg, v, a = pol.forward(torch.from_numpy(pack(obs)).cuda(), seed=seed, step=step)
    pol.sync()
    check_outputs(params, obs, lg, v)
    u = philox_u(seed, step, n)
    lgh = lg.cpu().numpy().astype(np.float64)
    want = P.sample(lgh, u)
    ok = P.cdf_margin(lgh, u) > MARGIN
    assert ok.mean() > 0.99
    assert np.array_equal(a.cpu().numpy()[ok], want[ok])
    assert len(np.unique(a.cpu().numpy())) > 1


def test_forward_full_size_sampled():
    """16,384 instances (128 conv batches per SM wave, 128 head tiles):
    sampled instances against the oracle."""
    o = octax()
    n, L = 16384, 5
    params = W.policy_params(4, L)
    obs = random_frames(n, 0.08, 44)
    pol = o.Policy(params, max_envs=n)
    lg, v, a = pol.forward(torch.from_numpy(pack(obs)).cuda(), seed=9, step=1)
    pol.sync()
    idx = np.unique(np.concatenate([np.random.default_rng(1).choice(n, 48, replace=False),
                                    [0, 7, 8, 127, 128, n - 129, n - 1]]))
    check_outputs(params, obs[idx], lg[idx], v[idx])


def test_rollout_teacher_forced():
    """The on-device rollout: the policy draws every action from its own
    logits, the environment steps with them. Replaying the drawn actions in
    the oracle environment gives bit-identical rewards, done flags and final
    observation; at every step the logits and value match the oracle network
    on the oracle's observation, and every draw is the inverse-CDF draw."""
    o = octax()
    g = W.template_game(W.TemplateParams(seed=3), score_limit=2, max_episode_steps=30)
    n, T, L = 200, 40, g.n_actions + 1
    params = W.policy_params(8, L)
    env = o.Env([g], n, seed=11)
    ref = oracle.OracleEnv([g], n, seed=11)
    obs0 = env.reset()
    o0 = ref.reset()
    assert np.array_equal(obs0.cpu().numpy(), o0)
    pol = o.Policy(params, max_envs=n)
    words = torch.from_numpy(pack(o0)).cuda()
    seed = 77
    a, lg, v, r, d = pol.rollout(env, T, words, seed=seed, step0=100)
    pol.sync()
    env.sync()
    a_h = a.cpu().numpy()
    cur = o0
    for k in range(T):
        l16 = check_outputs(params, cur, lg[k], v[k])
        u = philox_u(seed, 100 + k, n)
        lgk = lg[k].cpu().numpy().astype(np.float64)
        ok = P.cdf_margin(lgk, u) > MARGIN
        assert np.array_equal(a_h[k][ok], P.sample(lgk, u)[ok])
        ob, rw, dn = ref.step(a_h[k])
        assert np.array_equal(r[k].cpu().numpy(), rw), k
        assert np.array_equal(d[k].cpu().numpy(), dn), k
        cur = ob
    assert np.array_equal(words.cpu().numpy(), pack(cur))
    assert np.array_equal(env.state_hash().cpu().numpy().view(np.uint64), ref.hashes())
    assert int(d.sum()) > 0 and len(np.unique(a_h)) >= 3


def test_rollout_full_size_sampled():
    """The rollout the bench times: 16,384 instances of its template workload
    (seed 2), its network (weights seed 1, 5 logits) and seeds, default
    launch. Every instance's rewards, done flags, final observation and state
    hash match the oracle environment replaying the drawn actions; at every
    step sampled instances' logits, value and draw match the oracle network."""
    o = octax()
    w = W.cfg_scale(n_envs=16384)
    g = w.games[0]
    n, T, L = w.n_envs, 4, g.n_actions + 1
    params = W.policy_params(1, L)
    env = o.Env(w.games, n, seed=w.seed)
    ref = oracle.OracleEnv(w.games, n, seed=w.seed)
    o0 = ref.reset()
    assert np.array_equal(env.reset().cpu().numpy(), o0)
    pol = o.Policy(params, max_envs=n)
    words = torch.from_numpy(pack(o0)).cuda()
    a, lg, v, r, d = pol.rollout(env, T, words, seed=1, step0=0)
    pol.sync()
    env.sync()
    a_h = a.cpu().numpy()
    idx = np.unique(np.concatenate([np.random.default_rng(2).choice(n, 40, replace=False),
                                    [0, 7, 8, 127, 128, n - 129, n - 1]]))
    cur = o0
    for k in range(T):
        check_outputs(params, cur[idx], lg[k][idx], v[k][idx])
        u = philox_u(1, k, n, idx)
        lgk = lg[k].cpu().numpy()[idx].astype(np.float64)
        ok = P.cdf_margin(lgk, u) > MARGIN
        assert np.array_equal(a_h[k][idx][ok], P.sample(lgk, u)[ok])
        ob, rw, dn = ref.step(a_h[k])
        assert np.array_equal(r[k].cpu().numpy(), rw), k
        assert np.array_equal(d[k].cpu().numpy(), dn), k
        cur = ob
    assert np.array_equal(words.cpu().numpy(), pack(cur))
    assert np.array_equal(env.state_hash().cpu().numpy().view(np.uint64), ref.hashes())
    assert len(np.unique(a_h)) >= 3


def test_policy_rejects_bad_arguments():
    o = octax()
    params = W.policy_params(1, 5)
    bad = dict(params)
    bad["wa2"] = np.zeros((18, 256), np.float32)
    bad["ba2"] = np.zeros(18, np.float32)
    with pytest.raises(o.OctaxError):
        o.Policy(bad, max_envs=8)
    pol = o.Policy(params, max_envs=8)
    words = torch.zeros((9, 4, 32), dtype=torch.int64, device="cuda")
    with pytest.raises(o.OctaxError):
        pol.forward(words)
    g = W.template_game(W.TemplateParams(seed=1))
    env = o.Env([g], 16, seed=1)
    with pytest.raises(o.OctaxError):      # more instances than max_envs
        pol.rollout(env, 2, torch.zeros((16, 4, 32), dtype=torch.int64, device="cuda"))


def test_bounded_wait_failure_is_reported_and_recovered():
    """The conv kernel's waits are bounded: with its first completion signal
    withheld (octax_policy_debug_stall) the wait runs out after about a
    second, the kernel returns, octax_policy_sync reports OCTAX_ECUDA once,
    and the same policy then computes correct outputs again."""
    import time

    o = octax()
    n, L = 64, 5
    params = W.policy_params(21, L)
    obs = random_frames(n, 0.1, 21)
    pol = o.Policy(params, max_envs=n)
    words = torch.from_numpy(pack(obs)).cuda()
    pol.debug_stall(True)
    t0 = time.monotonic()
    pol.forward(words)
    with pytest.raises(o.OctaxError) as e:
        pol.sync()
    assert e.value.code == o.ECUDA
    assert time.monotonic() - t0 < 30
    pol.debug_stall(False)
    pol.sync()                                  # the report was cleared
    lg, v, _ = pol.forward(words)
    pol.sync()
    check_outputs(params, obs, lg, v)


def test_rollouts_chain_across_calls_and_games():
    """A rollout of 5 then one of 7 steps (step0 continuing) equals one of
    12 steps from the same start, bit for bit (actions, logits, values,
    rewards, done flags, final observation and state), in an environment
    that mixes two games with different K."""
    o = octax()
    g1 = W.template_game(W.TemplateParams(seed=5), score_limit=2, max_episode_steps=9)
    g2 = W.replace(W.template_game(W.TemplateParams(seed=6), max_episode_steps=7), instr_per_frame=15)
    n, L = 300, g1.n_actions + 1
    goe = (np.arange(n) % 2).astype(np.uint16)
    params = W.policy_params(31, L)
    pol = o.Policy(params, max_envs=n)
    outs = []
    for split in ((12,), (5, 7)):
        env = o.Env([g1, g2], n, seed=4, game_of_env=goe)
        words = pack_words_dev(env.reset())
        parts, step0 = [], 10
        for T in split:
            parts.append(pol.rollout(env, T, words, seed=9, step0=step0))
            step0 += T
        pol.sync()
        cat = [torch.cat([p[k] for p in parts]) for k in range(5)]
        outs.append((cat, words.clone(), env.state_hash().clone()))
    (a, w, h), (b, w2, h2) = outs
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert torch.equal(w, w2) and torch.equal(h, h2)
    assert int(a[4].sum()) > 0                   # episodes ended inside the rollouts


def pack_words_dev(obs):
    return (obs.to(torch.int64) << torch.arange(64, device=obs.device)).sum(dim=-1)


def test_rollout_rejects_unsupported_environments():
    o = octax()
    params = W.policy_params(2, 5)
    pol = o.Policy(params, max_envs=64)
    env = o.Env([W.schip_template_game(W.TemplateParams(seed=3))], 16, seed=1)
    with pytest.raises(o.OctaxError) as e:          # Super-CHIP frames are 64 x 128
        pol.rollout(env, 1, torch.zeros((16, 4, 32), dtype=torch.int64, device="cuda"))
    assert e.value.code == o.EINVAL
    g = W.replace(W.template_game(W.TemplateParams(seed=1)), stack_frames=2)
    env = o.Env([g], 16, seed=1)
    with pytest.raises(o.OctaxError) as e:
        pol.rollout(env, 1, torch.zeros((16, 4, 32), dtype=torch.int64, device="cuda"))
    assert e.value.code == o.EINVAL
