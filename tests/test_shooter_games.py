"""The Target Shooter levels (App. D) run on the oracle and behave as the
paper describes them: hits add one to V2, the game ends with V3 = 1 after ten
targets, level 2-3 targets expire, level 3 targets move. These tests pin the
ROMs (inputs); the GPU parity tests then run them on both sides."""
import numpy as np
import pytest

from paper_2510_01764_gb300 import workloads as W

NOOP = len(W.SHOOTER_KEYS)


def chase(V, tol=1):
    """Move the crosshair towards the target, shoot when within tol."""
    dx, dy = int(V[4]) - int(V[0]), int(V[5]) - int(V[1])
    if abs(dx) <= tol and abs(dy) <= tol:
        return 4
    if abs(dx) > abs(dy):
        return 3 if dx > 0 else 1
    return 2 if dy > 0 else 0


def to_loop(oracle_lib, level):
    m = oracle_lib.Machine(W.shooter_game(level), seed=3, uid=level)
    loop = W.shooter_labels(level)["loop"]
    for _ in range(200):
        if m.m.PC == loop:
            return m
        m.exec()
    raise AssertionError("init did not reach the main loop")


def test_descriptor_register_mapping():
    for level in (1, 2, 3):
        g = W.shooter_game(level)
        assert g.action_set == (5, 7, 8, 9, 6)
        assert g.score == (W.Term("reg", 2),)
        assert g.term == (W.Clause(W.Term("reg", 3), "==", 1),)


def test_init_state(oracle_lib):
    for level in (1, 2, 3):
        m = to_loop(oracle_lib, level)
        V = m.V
        assert (V[0], V[1], V[2], V[3], V[6]) == (30, 14, 0, 0, 1)
        assert 2 <= V[4] <= 57 and 2 <= V[5] <= 25
        # the crosshair, the target and the score glyph "0" are on screen
        assert m.pixels[14 + 2, 30:35].all() and m.pixels.sum() > 10
        if level >= 2:
            assert m.m.DT == (90 if level == 2 else 120)


@pytest.mark.parametrize("dx,dy", [(dx, dy) for dx in range(-3, 4) for dy in range(-3, 4)])
def test_hit_needs_the_crosshair_within_two_pixels(oracle_lib, dx, dy):
    m = to_loop(oracle_lib, 1)
    V = m.V
    m.set_V(0, (V[4] + dx) & 0xFF)
    m.set_V(1, (V[5] + dy) & 0xFF)
    m.exec(80, key=6)
    hit = abs(dx) <= 2 and abs(dy) <= 2
    assert (m.V[2] >= 1) == hit
    assert m.V[6] >= 2 if hit else m.V[6] == 1     # a hit shows the next target


def test_tenth_target_ends_the_game(oracle_lib):
    m = to_loop(oracle_lib, 1)
    m.set_V(6, 10)
    m.set_V(0, m.V[4])
    m.set_V(1, m.V[5])
    m.exec(100, key=6)
    end = W.shooter_labels(1)["end"]
    assert m.V[3] == 1 and m.V[2] == 1 and m.m.PC == end
    m.exec(50)
    assert m.m.PC == end and m.V[3] == 1


def test_scripted_policy_clears_level_one(oracle_lib):
    e = oracle_lib.OracleEnv([W.shooter_game(1)], 1, seed=1)
    e.reset()
    total = 0.0
    for step in range(600):
        _, r, d = e.step(np.array([chase(e.records()["V"][0])], np.uint8))
        assert r[0] in (0.0, 1.0)
        total += float(r[0])
        if d[0]:
            break
    assert d[0] == 1 and total == W.SHOOTER_TARGETS


def test_idle_player_scores_nothing(oracle_lib):
    """Level 1 targets wait forever; level 2-3 targets expire, ten of them
    end the game after about ten lifetimes."""
    for level, life in ((1, None), (2, 90), (3, 120)):
        e = oracle_lib.OracleEnv([W.shooter_game(level)], 1, seed=level)
        e.reset()
        _, r, d, _ = e.rollout(np.full((1000, 1), NOOP, np.uint8))
        assert r.sum() == 0
        if life is None:
            assert d.sum() == 0
        else:
            first = int(np.argmax(d[:, 0]))
            assert d[first, 0] == 1
            assert 10 * life // 4 <= first + 1 <= 10 * life // 4 + 12


def test_level_three_targets_move_and_bounce(oracle_lib):
    m = oracle_lib.Machine(W.shooter_game(3), seed=9, uid=1)
    xs, ys, ns = [], [], []
    for _ in range(280):
        m.step(NOOP, obs=False)
        xs.append(m.V[4])
        ys.append(m.V[5])
        ns.append(m.V[6])
    xs, ys, ns = map(np.array, (xs, ys, ns))
    # a step may end inside the respawn code; keep steps with no respawn
    # started before the next one
    settled = np.r_[ns[1:] == ns[:-1], False]
    assert xs[settled].min() >= 2 and xs[settled].max() <= 57
    assert ys[settled].min() >= 2 and ys[settled].max() <= 25
    pair = settled[:-1] & settled[1:] & (ns[1:] == ns[:-1])
    moved = (xs[1:] != xs[:-1]) | (ys[1:] != ys[:-1])
    assert pair.sum() > 200 and moved[pair].mean() > 0.5
    assert np.abs(np.diff(xs))[pair].max() <= 4 and np.abs(np.diff(ys))[pair].max() <= 4
    assert ns[-1] >= 9


def test_chase_beats_random_on_every_level(oracle_lib):
    for level in (1, 2, 3):
        n = 8
        e = oracle_lib.OracleEnv([W.shooter_game(level)], n, seed=level)
        e.reset()
        scripted = 0.0
        for _ in range(300):
            V = e.records()["V"]
            _, r, _ = e.step(np.array([chase(V[i]) for i in range(n)], np.uint8))
            scripted += float(r.sum())
        e2 = oracle_lib.OracleEnv([W.shooter_game(level)], n, seed=level)
        e2.reset()
        _, r2, _, _ = e2.rollout(W.actions(level, 0, 300, n, 5))
        assert scripted > 4 * max(float(r2.sum()), 1.0)
