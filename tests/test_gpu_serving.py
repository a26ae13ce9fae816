"""Continuous-batching server: every request's result is bit-identical alone
and in a mix (and to a plain environment and the oracle with the same seed),
admission respects the memory budget, and bookkeeping errors are reported."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2510_01764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SLOT_BYTES = 4476 + 8  # >= per-slot state (4,468 B) + step buffers (8 B): k * SLOT_BYTES holds >= k slots


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


def games():
    g = W.cfg_batch(n_envs=64, n_steps=1).games[:6]
    return g + [W.replace(W.random_game(3), action_set=g[0].action_set)]


def make_requests(k, seed, max_envs=700):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(k):
        n = int(np.exp(rng.uniform(0, np.log(max_envs))))
        T = int(rng.integers(1, 9))
        game = int(rng.integers(0, 7))
        acts = rng.integers(0, 5, size=(T, n), dtype=np.uint8)
        reqs.append(dict(game=game, actions=acts, seed=int(rng.integers(0, 2**63))))
    return reqs


def run_all(server, reqs, stagger_s=0.0):
    ids = []
    for r in reqs:
        ids.append(server.submit(r["game"], r["actions"], r["seed"]))
        if stagger_s:
            time.sleep(stagger_s)
    infos = [server.wait(i, timeout_ms=60000) for i in ids]
    outs = [tuple(t.cpu() for t in server.outputs(i)) for i in ids]
    return ids, infos, outs


def test_alone_equals_in_mix():
    o = octax()
    gs = games()
    reqs = make_requests(40, 1)
    total = sum(r["actions"].shape[1] for r in reqs)
    # budget for about a third of all instances: admission has to queue
    srv = o.Server(gs, memory_budget_bytes=(total // 3) * SLOT_BYTES, block=64, inst_per_warp=8)
    _, infos, mixed = run_all(srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["peak_active_envs"] <= st["slots_capacity"]
    assert st["peak_active_requests"] > 1          # requests shared launches
    assert any(i["admit_ns"] - i["submit_ns"] > 0 for i in infos)
    srv.close()
    # each request alone on a fresh server, and through a plain environment
    for r, got in list(zip(reqs, mixed))[::3]:
        solo = o.Server(gs, memory_budget_bytes=4096 * SLOT_BYTES, block=128, inst_per_warp=32)
        _, _, alone = run_all(solo, [r])
        solo.close()
        for x, y in zip(got, alone[0]):
            assert torch.equal(x, y)
        T, n = r["actions"].shape
        env = o.Env(gs, n, seed=r["seed"], game_of_env=np.full(n, r["game"], np.uint16))
        e_obs, e_rew, e_done = env.step_n(torch.from_numpy(r["actions"]).cuda())
        assert torch.equal(got[0], e_obs.cpu()) and torch.equal(got[1], e_rew.cpu())
        assert torch.equal(got[2], e_done.cpu())
        env.close()


@pytest.mark.parametrize("shape", [None, (64, 1), (32, 2), (128, 4)])
def test_requests_match_oracle(shape):
    """Requests against the oracle, with the server's default CTA shape and
    with warps of 1, 2 and 4 instances (whose frames all 32 lanes write)."""
    o = octax()
    gs = games()
    reqs = make_requests(6, 2, max_envs=64)
    kw = {} if shape is None else dict(block=shape[0], inst_per_warp=shape[1])
    srv = o.Server(gs, memory_budget_bytes=10000 * SLOT_BYTES, **kw)
    _, _, outs = run_all(srv, reqs, stagger_s=0.0005)
    srv.close()
    for r, got in zip(reqs, outs):
        T, n = r["actions"].shape
        ref = oracle.OracleEnv(gs, n, seed=r["seed"], game_of_env=np.full(n, r["game"], np.uint16))
        ref.reset()
        ob, rw, dn, _ = ref.rollout(r["actions"], obs=True)
        assert np.array_equal(got[0].numpy(), ob)
        assert np.array_equal(got[1].numpy(), rw)
        assert np.array_equal(got[2].numpy(), dn)


def test_requests_with_wrappers_match_oracle():
    """Sticky actions and no-op reset (§3.2) through the serving path."""
    o = octax()
    gs = games()
    gs[1] = W.replace(gs[1], sticky_prob=0.3, max_noops=9)
    gs[4] = W.replace(gs[4], max_noops=3)
    reqs = make_requests(6, 5, max_envs=64)
    srv = o.Server(gs, memory_budget_bytes=10000 * SLOT_BYTES)
    _, _, outs = run_all(srv, reqs, stagger_s=0.0005)
    srv.close()
    for r, got in zip(reqs, outs):
        n = r["actions"].shape[1]
        ref = oracle.OracleEnv(gs, n, seed=r["seed"], game_of_env=np.full(n, r["game"], np.uint16))
        ref.reset()
        ob, rw, dn, _ = ref.rollout(r["actions"], obs=True)
        assert np.array_equal(got[0].numpy(), ob)
        assert np.array_equal(got[1].numpy(), rw)
        assert np.array_equal(got[2].numpy(), dn)


def test_poisson_arrivals_from_threads():
    """Requests submitted from two threads at random times all complete, and
    the ones that overlapped in time were batched together."""
    o = octax()
    gs = games()
    srv = o.Server(gs, memory_budget_bytes=3000 * SLOT_BYTES)
    reqs = make_requests(60, 3, max_envs=300)
    ids = [None] * len(reqs)
    rng = np.random.default_rng(4)

    def worker(part):
        for k in part:
            time.sleep(float(rng.exponential(0.0005)))
            r = reqs[k]
            ids[k] = srv.submit(r["game"], r["actions"], r["seed"])

    ths = [threading.Thread(target=worker, args=(range(i, len(reqs), 2),)) for i in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    lat = []
    for i in ids:
        info = srv.wait(i, timeout_ms=60000)
        assert info["state"] == 2 and info["done_ns"] >= info["admit_ns"] >= info["submit_ns"]
        lat.append((info["done_ns"] - info["submit_ns"]) / 1e6)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["env_steps"] == sum(int(np.prod(r["actions"].shape)) for r in reqs)
    for i in ids:
        srv.release(i)
    srv.close()
    assert max(lat) < 10000


def test_server_errors():
    o = octax()
    gs = games()
    srv = o.Server(gs, memory_budget_bytes=100 * SLOT_BYTES)
    with pytest.raises(o.OctaxError) as e:
        srv.submit(0, np.zeros((1, 101), np.uint8), 1)      # larger than the pool
    assert e.value.code == o.ENOMEM
    with pytest.raises(o.OctaxError) as e:
        srv.submit(0, np.zeros((9, 4), np.uint8), 1)        # too many steps
    assert e.value.code == o.EINVAL
    with pytest.raises(o.OctaxError) as e:
        srv.submit(99, np.zeros((1, 4), np.uint8), 1)       # unknown game
    assert e.value.code == o.EINVAL
    with pytest.raises(o.OctaxError) as e:
        srv.wait(12345, timeout_ms=10)
    assert e.value.code == o.ENOTFOUND
    rid = srv.submit(0, np.zeros((2, 100), np.uint8), 1)
    srv.wait(rid)
    srv.release(rid)
    with pytest.raises(o.OctaxError):
        srv.query(rid)
    srv.close()


def test_batched_submit_equals_single_submits():
    """octax_server_submit_batch / octax_server_wait_batch: the same requests
    queued in one call give the same outputs as queued one by one, the infos
    come back in order and released ids are forgotten; an invalid request in
    a batch queues nothing."""
    o = octax()
    gs = games()
    reqs = make_requests(24, 7, max_envs=500)
    total = sum(r["actions"].shape[1] for r in reqs)
    srv = o.Server(gs, memory_budget_bytes=(total // 2) * SLOT_BYTES, block=128, inst_per_warp=16)
    _, _, single = run_all(srv, reqs)
    items = []
    for r in reqs:
        T, n = r["actions"].shape
        out = (torch.empty((T, n, 4, 32, 64), dtype=torch.uint8, device="cuda"),
               torch.empty((T, n), dtype=torch.float32, device="cuda"),
               torch.empty((T, n), dtype=torch.uint8, device="cuda"))
        items.append((r["game"], r["actions"], r["seed"], out))
    ids = srv.submit_batch(items)
    assert ids == sorted(ids) and len(set(ids)) == len(ids)
    infos = srv.wait_batch(ids, release=True, timeout_ms=60000)
    assert all(i["state"] == 2 and i["done_ns"] >= i["admit_ns"] >= i["submit_ns"] for i in infos)
    for (_, _, _, out), want in zip(items, single):
        for x, y in zip(out, want):
            assert torch.equal(x.cpu(), y)
    with pytest.raises(o.OctaxError) as e:
        srv.query(ids[0])
    assert e.value.code == o.ENOTFOUND
    bad = list(items[:2]) + [(99, items[2][1], 1, items[2][3])]
    before = srv.stats()["submitted"]
    with pytest.raises(o.OctaxError):
        srv.submit_batch(bad)
    assert srv.stats()["submitted"] == before
    srv.close()


def test_lone_request_takes_one_launch():
    """A request that runs alone advances all its steps in one tick (the
    tick takes the fewest steps any running request has left), with the
    oracle's results; a mix still matches the oracle step by step."""
    o = octax()
    gs = games()
    srv = o.Server(gs, memory_budget_bytes=5000 * SLOT_BYTES)
    rng = np.random.default_rng(9)
    acts = rng.integers(0, 5, size=(8, 300), dtype=np.uint8)
    ids, _, outs = run_all(srv, [dict(game=2, actions=acts, seed=77)])
    st = srv.stats()
    assert st["ticks"] == 1 and st["env_steps"] == 8 * 300
    ref = oracle.OracleEnv(gs, 300, seed=77, game_of_env=np.full(300, 2, np.uint16))
    ref.reset()
    ob, rw, dn, _ = ref.rollout(acts, obs=True)
    assert np.array_equal(outs[0][0].numpy(), ob)
    assert np.array_equal(outs[0][1].numpy(), rw)
    assert np.array_equal(outs[0][2].numpy(), dn)
    srv.close()
