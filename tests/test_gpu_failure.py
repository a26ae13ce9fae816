"""Failure path of the warp-specialised kernel, exercised without a GPU fault:
the writer warps are told to skip their hand-over (a barrier phase that
nothing completes), so the emulator warps' bounded waits run out after about
a second, the kernel records the failure and returns, octax_sync reports it
once, and the environment — its state untouched by the failed launch — goes
on stepping bit-exactly."""
import time

import numpy as np
import pytest

import oracle
from paper_2510_01764_gb300 import workloads as W
from test_gpu_parity import hashes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_01764_gb300 import build

    build.build()
    oracle.build()


def test_stalled_hand_over_is_reported_and_the_env_recovers():
    from paper_2510_01764_gb300 import octax as o

    g = W.template_game(W.TemplateParams(seed=4), score_limit=3)
    n = 2048
    env = o.Env([g], n, seed=5)
    env.set_launch(block=128, inst_per_warp=16, steps_per_launch=4, persistent=0, use_graph=0,
                   writer_warps=2)
    h0 = hashes(env)
    acts = W.actions(5, 0, 8, n, 5)
    a_dev = torch.from_numpy(acts).cuda()

    env.debug_stall_writers(True)
    t0 = time.monotonic()
    env.step_n(a_dev[:4])
    with pytest.raises(o.OctaxError) as ei:
        env.sync()
    elapsed = time.monotonic() - t0
    assert ei.value.code == o.ECUDA and "timed out" in str(ei.value)
    assert elapsed < 20.0
    assert np.array_equal(hashes(env), h0)       # the failed launch stored no state
    env.sync()                                    # reported once, then cleared

    env.debug_stall_writers(False)
    obs, rew, done = env.step_n(a_dev)
    env.sync()
    ref = oracle.OracleEnv([g], n, seed=5)
    o2, r2, d2, _ = ref.rollout(acts, obs=True)
    assert np.array_equal(obs.cpu().numpy(), o2)
    assert np.array_equal(rew.cpu().numpy(), r2)
    assert np.array_equal(done.cpu().numpy(), d2)
    assert np.array_equal(hashes(env), ref.hashes())
