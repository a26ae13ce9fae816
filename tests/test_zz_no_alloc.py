"""octax_rollout_static: the entry point for callers that may not allocate
device memory (code inside another framework's memory pool, plugins whose
host forbids allocation after start-up, real-time loops that cannot afford
an allocation's synchronisation). It keeps all scratch state in a static
device array; its results must equal octax_create + octax_step_n exactly,
call after call, although each call reuses the array the previous call left
behind.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2510_01764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_01764_gb300 import build

    build.build()
    oracle.build()


def rollout_static(game, n, seed, actions, quirks=0):
    from paper_2510_01764_gb300 import octax as o

    L = o.load_library()
    T = actions.shape[0]
    obs = torch.full((T, n, game.stack_frames, 32, 64), 7, dtype=torch.uint8, device="cuda")
    rew = torch.full((T, n), -1.0, dtype=torch.float32, device="cuda")
    done = torch.full((T, n), 7, dtype=torch.uint8, device="cuda")
    cg, keep = o.make_game(game)
    stream = torch.cuda.current_stream()
    rc = L.octax_rollout_static(C.byref(cg), n, quirks, seed, T, C.c_void_p(actions.data_ptr()),
                                C.c_void_p(obs.data_ptr()), C.c_void_p(rew.data_ptr()),
                                C.c_void_p(done.data_ptr()), C.c_void_p(stream.cuda_stream))
    o.check(rc)
    torch.cuda.synchronize()
    del keep
    return obs, rew, done


def reference(game, n, seed, actions, quirks=0):
    from paper_2510_01764_gb300 import octax as o

    env = o.Env([game], n, seed=seed, quirks=quirks)
    out = env.step_n(actions)
    torch.cuda.synchronize()
    env.close()
    return out


def test_static_rollout_matches_step_n_twice_in_a_row():
    cases = [
        (W.template_game(W.TemplateParams(seed=2), score_limit=3, max_episode_steps=40), 1000, 11, 90),
        (W.random_game(5), 77, 12, 33),        # fewer instances: stale state must not leak
        (W.replace(W.template_game(W.TemplateParams(seed=4), max_episode_steps=12), sticky_prob=0.25,
                   max_noops=6), 300, 13, 40),  # sticky actions + no-op reset
    ]
    for game, n, seed, T in cases:
        acts = torch.from_numpy(W.actions(seed, 0, T, n, game.n_actions + 1)).cuda()
        got = rollout_static(game, n, seed, acts)
        ref = reference(game, n, seed, acts)
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
    assert int(got[2].sum()) >= 0


def test_static_rollout_at_capacity_matches_step_n_and_oracle():
    """Exactly 1,024 instances (the last CTA group full, every state array
    used to its end), twice in a row; the second call is also checked
    against the CPU oracle directly."""
    game = W.template_game(W.TemplateParams(seed=6), score_limit=2, max_episode_steps=25)
    n, seed, T = 1024, 21, 48
    for rep in range(2):
        acts = torch.from_numpy(W.actions(seed + rep, 0, T, n, game.n_actions + 1)).cuda()
        got = rollout_static(game, n, seed, acts)
        ref = reference(game, n, seed, acts)
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
    orc = oracle.OracleEnv([game], n, seed=seed)
    orc.reset()
    o2, r2, d2, _ = orc.rollout(acts.cpu().numpy(), obs=True)
    assert np.array_equal(got[0].cpu().numpy(), o2)
    assert np.array_equal(got[1].cpu().numpy(), r2)
    assert np.array_equal(got[2].cpu().numpy(), d2)
    assert int(got[2].sum()) > 0


def test_static_rollout_rejects_oversize():
    from paper_2510_01764_gb300 import octax as o

    game = W.template_game(W.TemplateParams(seed=1))
    acts = torch.zeros((1, 1025), dtype=torch.uint8, device="cuda")
    with pytest.raises(o.OctaxError) as e:
        rollout_static(game, 1025, 1, acts)
    assert e.value.code == o.EINVAL
