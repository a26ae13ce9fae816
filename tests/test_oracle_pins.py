"""Pins of the CPU oracle to facts outside itself.

Each test checks the oracle against something the paper or mathematics fixes:
published known-answer vectors, the memory map (App. B), closed forms and
invariants (XOR-twice-erases, carry/borrow identities, BCD), hand-assembled
programs whose results follow from integer arithmetic (16-bit add/sub,
shift-and-add multiply), the paper's own score/termination expressions
(§3.3, App. C) and brute force over all 8-bit operand pairs.
"""
import os

import numpy as np
import pytest

from chip8_prog import PAPER_EXPR, PAPER_GAMES, prog
from paper_2510_01764_gb300.workloads import Clause, GameSpec, Term

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def machine(oracle, words, data=b"", quirks=0, seed=0, uid=0, **kw):
    return oracle.Machine(prog(words, data, **kw), quirks=quirks, seed=seed, uid=uid)


# ---------------------------------------------------------------- RNG / hash
def test_philox_known_answers(oracle_lib):
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = [int(t, 16) for t in line.split()]
        assert oracle_lib.philox4x32_10(f[0:4], f[4:6]) == tuple(f[6:10])


def test_fnv1a64_vectors(oracle_lib):
    for line in open(os.path.join(GOLD, "fnv1a64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        data, h = line.split()
        b = b"" if data == "-" else bytes.fromhex(data)
        assert oracle_lib.fnv1a64(b) == int(h, 16)


# ---------------------------------------------------------------- memory map
def test_reset_memory_map(oracle_lib):
    """App. B / §3.2: 4 KB, program at 0x200, font at 0x050-0x09F, PC = 0x200."""
    code = bytes(range(1, 200))
    m = oracle_lib.Machine(GameSpec(rom=code))
    ram = m.ram
    assert ram.shape == (4096,)
    assert bytes(ram[0x200:0x200 + len(code)]) == code
    assert m.m.PC == 0x200 and m.m.I == 0 and m.m.SP == 0
    font = ram[0x50:0xA0]
    assert np.all(ram[:0x50] == 0) and np.all(ram[0xA0:0x200] == 0)
    assert np.all(ram[0x200 + len(code):] == 0)
    # 16 glyphs x 5 bytes, each 4 pixels wide (low nibble clear), none blank
    glyphs = font.reshape(16, 5)
    assert np.all((glyphs & 0x0F) == 0)
    assert all(g.any() for g in glyphs)
    assert len({bytes(g) for g in glyphs}) == 16
    assert np.all(m.pixels == 0)
    assert m.V == [0] * 16


def test_fx29_font_address(oracle_lib):
    """App. B "Font System": glyph d at 0x050 + 5 d (5-byte stride)."""
    for v in range(256):
        m = machine(oracle_lib, [0xF329])
        m.set_V(3, v)
        m.exec()
        assert m.m.I == 0x50 + 5 * (v % 16)


def test_rom_size_limit(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.OracleEnv([GameSpec(rom=b"\x00" * 3585)], 1)
    oracle_lib.OracleEnv([GameSpec(rom=b"\x00" * 3584)], 1)


# ---------------------------------------------------------------- ALU brute force
def _alu_all_pairs(oracle, op):
    """Run ``op`` (X = 0, Y = 1) for all 65,536 (a, b); VF preset to 0xAA."""
    m = machine(oracle, [op])
    out = np.zeros((256, 256, 2), dtype=np.int64)
    for a in range(256):
        for b in range(256):
            m.m.PC = 0x200
            m.m.V[0] = a
            m.m.V[1] = b
            m.m.V[15] = 0xAA
            m.exec()
            out[a, b, 0] = m.m.V[0]
            out[a, b, 1] = m.m.V[15]
    return out


A, B = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")


def test_alu_add_carry_all_pairs(oracle_lib):
    """8XY4: the carry flag and the 8-bit sum recompose the integer sum."""
    r = _alu_all_pairs(oracle_lib, 0x8014)
    assert np.all(256 * r[..., 1] + r[..., 0] == A + B)
    assert set(np.unique(r[..., 1])) <= {0, 1}


def test_alu_sub_borrow_all_pairs(oracle_lib):
    """8XY5 / 8XY7: VF = 1 exactly when the difference is non-negative."""
    r = _alu_all_pairs(oracle_lib, 0x8015)
    assert np.all((r[..., 0] + B) % 256 == A)
    assert np.all(r[..., 1] == (A - B >= 0))
    r = _alu_all_pairs(oracle_lib, 0x8017)
    assert np.all((r[..., 0] + A) % 256 == B)
    assert np.all(r[..., 1] == (B - A >= 0))


def test_alu_shifts_all_pairs(oracle_lib):
    """8XY6 / 8XYE shift VX (fixed quirk set) and expose the bit shifted out."""
    r = _alu_all_pairs(oracle_lib, 0x8016)
    assert np.all(2 * r[..., 0] + r[..., 1] == A)
    r = _alu_all_pairs(oracle_lib, 0x801E)
    assert np.all(r[..., 0] + 256 * r[..., 1] == 2 * A)


def test_alu_logic_and_moves_all_pairs(oracle_lib):
    """8XY0-8XY3 against numpy's bitwise ops; VF untouched."""
    for op, ref in ((0x8010, B), (0x8011, np.bitwise_or(A, B)), (0x8012, np.bitwise_and(A, B)),
                    (0x8013, np.bitwise_xor(A, B))):
        r = _alu_all_pairs(oracle_lib, op)
        assert np.all(r[..., 0] == ref)
        assert np.all(r[..., 1] == 0xAA)


def test_add_immediate_all_values(oracle_lib):
    """7XNN wraps modulo 256 and leaves VF alone."""
    for nn in (0, 1, 0x7F, 0x80, 0xFF):
        m = machine(oracle_lib, [0x7000 | nn])
        for a in range(256):
            m.m.PC = 0x200
            m.m.V[0] = a
            m.m.V[15] = 0xAA
            m.exec()
            assert (m.m.V[0] - nn) % 256 == a
            assert m.m.V[15] == 0xAA


def test_flag_register_as_destination(oracle_lib):
    """With X = F the flag is written last and wins (8FY4, 8FY5, 8FY6, 8FYE)."""
    for op, a, b, vf in ((0x8F14, 200, 100, 1), (0x8F14, 1, 2, 0), (0x8F15, 5, 3, 1),
                         (0x8F15, 3, 5, 0), (0x8F16, 3, 0, 1), (0x8F1E, 0x80, 0, 1),
                         (0x8F17, 5, 3, 0)):
        m = machine(oracle_lib, [op])
        m.m.V[15] = a
        m.m.V[1] = b
        m.exec()
        assert m.m.V[15] == vf


ADD16 = [0x8134, 0x80F4, 0x8024, 0x1206]
SUB16 = [0x8135, 0x6E01, 0x8EF5, 0x8025, 0x80E5, 0x120A]


@pytest.mark.parametrize("words,fn", [(ADD16, lambda a, b: (a + b) % 65536),
                                      (SUB16, lambda a, b: (a - b) % 65536)])
def test_multibyte_arithmetic_programs(oracle_lib, words, fn):
    """16-bit add / subtract built from 8XY4 carries and 8XY5 borrows."""
    rng = np.random.default_rng(0)
    pairs = [(0, 0), (0xFFFF, 1), (0x00FF, 0x0001), (0x1234, 0xFEDC), (0, 1), (0x8000, 0x8000)]
    pairs += [tuple(int(v) for v in rng.integers(0, 65536, 2)) for _ in range(300)]
    m = machine(oracle_lib, words)
    for a, b in pairs:
        for i in range(16):
            m.m.V[i] = 0
        m.m.PC = 0x200
        m.m.V[0], m.m.V[1], m.m.V[2], m.m.V[3] = a >> 8, a & 255, b >> 8, b & 255
        m.exec(len(words))
        assert (m.m.V[0] << 8 | m.m.V[1]) == fn(a, b)


# multiply V0 x V1 -> V2:V3 by shift-and-add (8XY6, 8XYE, 8XY4, 8XY1, skips, calls)
MUL8 = [
    0x6200, 0x6300, 0x6400, 0x8500, 0x6608,   # 0x200..0x208 init
    0x8106, 0x3F00, 0x2222,                   # 0x20A loop: V1 >>= 1; if bit: call add
    0x855E, 0x8EF0, 0x844E, 0x84E1,           # V4:V5 <<= 1
    0x76FF, 0x3600, 0x120A,                   # counter
    0x1220,                                   # 0x21E... end (self loop at 0x220)
    0x1220,
    0x8354, 0x82F4, 0x8244, 0x00EE,           # 0x222 add: V2:V3 += V4:V5
]


def test_shift_and_add_multiply_program(oracle_lib):
    rng = np.random.default_rng(1)
    pairs = [(0, 0), (255, 255), (1, 255), (255, 1), (16, 16), (3, 85)]
    pairs += [tuple(int(v) for v in rng.integers(0, 256, 2)) for _ in range(200)]
    m = machine(oracle_lib, MUL8)
    for a, b in pairs:
        m2 = machine(oracle_lib, MUL8)
        m2.m.V[0], m2.m.V[1] = a, b
        m2.exec(400)
        assert m2.m.PC == 0x220
        assert (m2.m.V[2] << 8 | m2.m.V[3]) == a * b, (a, b)
        assert m2.m.SP == 0 and m2.m.status == 0
    del m


# ---------------------------------------------------------------- BCD / bulk memory
def test_bcd_all_values(oracle_lib):
    """FX33 (App. B): decimal digits of VX; 255 -> 2, 5, 5; I unchanged."""
    for v in range(256):
        m = machine(oracle_lib, [0xA300, 0xF533])
        m.set_V(5, v)
        m.exec(2)
        d = m.ram[0x300:0x303]
        assert all(x < 10 for x in d)
        assert 100 * int(d[0]) + 10 * int(d[1]) + int(d[2]) == v
        assert m.m.I == 0x300
        if v == 255:
            assert list(d) == [2, 5, 5]


def test_store_load_roundtrip(oracle_lib):
    """FX55 then FX65 restore V0..VX; I unchanged (fixed quirk set)."""
    for x in range(16):
        m = machine(oracle_lib, [0xA400, 0xF055 | x << 8, 0xF065 | x << 8])
        vals = [(37 * i + 11) % 256 for i in range(16)]
        for i in range(16):
            m.set_V(i, vals[i])
        m.exec(2)
        assert list(m.ram[0x400:0x400 + x + 1]) == vals[:x + 1]
        assert m.ram[0x400 + x + 1] == 0
        for i in range(16):
            m.set_V(i, 0)
        m.exec()
        assert m.V[:x + 1] == vals[:x + 1]
        assert all(v == 0 for v in m.V[x + 1:])
        assert m.m.I == 0x400


def test_memory_addresses_wrap(oracle_lib):
    m = machine(oracle_lib, [0xAFFE, 0xF233])
    m.set_V(2, 123)
    m.exec(2)
    ram = m.ram
    assert (ram[0xFFE], ram[0xFFF], ram[0x000]) == (1, 2, 3)


# ---------------------------------------------------------------- display
SPRITE = bytes((0xF0, 0x90, 0xA5, 0xFF, 0x01))


def test_draw_twice_erases(oracle_lib):
    """App. B: drawing the same sprite twice erases it; the 2nd draw sets VF."""
    n_lit = sum(bin(b).count("1") for b in SPRITE)
    for x, y in ((0, 0), (10, 7), (56, 27), (33, 20)):
        m = machine(oracle_lib, [0xA20A, 0xD015, 0xD015, 0x1206, 0x0000], data=SPRITE)
        m.set_V(0, x)
        m.set_V(1, y)
        m.exec(2)
        assert m.m.V[15] == 0
        assert int(m.pixels.sum()) == n_lit
        for r, b in enumerate(SPRITE):
            for c in range(8):
                assert m.pixels[y + r, x + c] == (b >> (7 - c)) & 1
        m.exec(1)
        assert m.m.V[15] == 1
        assert m.pixels.sum() == 0


def test_draw_clips_at_edges_and_wraps_start(oracle_lib):
    full = bytes([0xFF] * 5)
    m = machine(oracle_lib, [0xA206, 0xD015, 0x1204], data=full)
    m.set_V(0, 60)
    m.set_V(1, 30)
    m.exec(2)
    assert m.pixels.sum() == 4 * 2 and m.pixels[30:32, 60:64].all()
    m = machine(oracle_lib, [0xA206, 0xD015, 0x1204], data=full, quirks=0x10)
    m.set_V(0, 60)
    m.set_V(1, 30)
    m.exec(2)
    assert m.pixels.sum() == 40 and m.pixels[0:3, 0:4].all()
    m = machine(oracle_lib, [0xA206, 0xD015, 0x1204], data=full)
    m.set_V(0, 64 + 5)
    m.set_V(1, 32 + 3)
    m.exec(2)
    assert m.pixels[3:8, 5:13].all() and m.pixels.sum() == 40


def test_collision_only_on_overlap(oracle_lib):
    m = machine(oracle_lib, [0xA20C, 0xD015, 0xD235, 0xD455, 0x1208, 0x0000], data=SPRITE)
    m.set_V(0, 0); m.set_V(1, 0)   # first
    m.set_V(2, 8); m.set_V(3, 0)   # disjoint (right)
    m.set_V(4, 4); m.set_V(5, 3)   # overlaps row 3 of the first
    m.exec(2)
    assert m.m.V[15] == 0
    m.exec(1)
    assert m.m.V[15] == 0
    m.exec(1)
    assert m.m.V[15] == 1


def test_draw_zero_rows_and_vf_coordinates(oracle_lib):
    m = machine(oracle_lib, [0xA208, 0xD010, 0x1204, 0x0000], data=SPRITE)
    m.m.V[15] = 1
    m.exec(2)
    assert m.m.V[15] == 0 and m.pixels.sum() == 0
    m = machine(oracle_lib, [0xA208, 0xDFE1, 0x1204, 0x0000], data=bytes([0x80]))
    m.m.V[15] = 9
    m.m.V[14] = 4
    m.exec(2)
    assert m.pixels[4, 9] == 1 and m.pixels.sum() == 1


def test_clear_screen(oracle_lib):
    m = machine(oracle_lib, [0xA208, 0xD015, 0x00E0, 0x1206], data=SPRITE)
    m.set_V(0, 3)
    m.exec(2)
    assert m.pixels.sum() > 0
    m.exec()
    assert m.pixels.sum() == 0


# ---------------------------------------------------------------- control flow
def test_jumps_and_skips(oracle_lib):
    m = machine(oracle_lib, [0x1ABC])
    m.exec()
    assert m.m.PC == 0xABC
    m = machine(oracle_lib, [0xBFFF])
    m.set_V(0, 2)
    m.exec()
    assert m.m.PC == 0x001
    cases = [(0x3005, 5, 0, True), (0x3005, 6, 0, False), (0x4005, 5, 0, False),
             (0x4005, 6, 0, True), (0x5010, 7, 7, True), (0x5010, 7, 8, False),
             (0x9010, 7, 7, False), (0x9010, 7, 8, True)]
    for op, v0, v1, skip in cases:
        m = machine(oracle_lib, [op])
        m.set_V(0, v0)
        m.set_V(1, v1)
        m.exec()
        assert m.m.PC == (0x204 if skip else 0x202), hex(op)


def test_nested_calls_sixteen_deep(oracle_lib):
    """2NNN/00EE: 16 nested calls return in order; the 17th overflows."""
    def build(depth):
        words = [0x2300, 0x1202]  # main: call sub0; halt at 0x202
        data = bytearray(0x300 - 0x204)
        subs = []
        for i in range(depth):
            nxt = 0x300 + 6 * (i + 1)
            subs += [0x7001, (0x2000 | nxt) if i + 1 < depth else 0x0000, 0x00EE]
        return words, bytes(data) + b"".join(bytes((w >> 8, w & 255)) for w in subs)
    words, data = build(16)
    m = machine(oracle_lib, words, data=data)
    max_sp = 0
    for _ in range(200):
        m.exec()
        max_sp = max(max_sp, m.m.SP)
    assert m.m.PC == 0x202 and m.m.SP == 0 and m.m.V[0] == 16 and max_sp == 16
    assert m.m.status == 0
    words, data = build(17)
    m = machine(oracle_lib, words, data=data)
    m.exec(300)
    assert m.m.status & oracle_lib.ST_STACK_FAULT


def test_return_on_empty_stack_faults(oracle_lib):
    m = machine(oracle_lib, [0x00EE])
    m.exec()
    assert m.m.status == oracle_lib.ST_STACK_FAULT and m.m.SP == 15 and m.m.PC == 0


def test_invalid_opcodes_flag_and_skip(oracle_lib):
    for op in (0x8018, 0x801F, 0x5011, 0x9012, 0xE000, 0xE19F, 0xF0FF, 0xF001):
        m = machine(oracle_lib, [op])
        before = m.V
        m.exec()
        assert m.m.status == oracle_lib.ST_BAD_OP, hex(op)
        assert m.m.PC == 0x202 and m.V == before
    for op in (0x0000, 0x0123, 0x0FFF):     # 0NNN: ignored machine-code call
        m = machine(oracle_lib, [op])
        m.exec()
        assert m.m.status == 0 and m.m.PC == 0x202


def test_index_register_ops(oracle_lib):
    m = machine(oracle_lib, [0xA123, 0xF41E, 0x1204])
    m.set_V(4, 0xFE)
    m.m.V[15] = 7
    m.exec(2)
    assert m.m.I == 0x123 + 0xFE and m.m.V[15] == 7
    m = machine(oracle_lib, [0xAFF0, 0xF41E], quirks=0x20)
    m.set_V(4, 0x20)
    m.exec(2)
    assert m.m.I == 0x1010 and m.m.V[15] == 1


# ---------------------------------------------------------------- timers and keys
def test_delay_and_sound_timers(oracle_lib):
    """60 Hz timers: set N, read back N - f after f frames, stop at 0."""
    m = machine(oracle_lib, [0x6005, 0xF015, 0xF018, 0xF107, 0x1206])
    m.exec(3)
    for f in range(8):
        assert m.m.DT == max(5 - f, 0) and m.m.ST == max(5 - f, 0)
        m.m.PC = 0x206
        m.exec()
        m.m.PC = 0x206
        m.tick()
    g = prog([0x6009, 0xF015, 0xF018, 0xF107, 0x1206], instr_per_frame=10, frameskip=4)
    mm = oracle_lib.Machine(g)
    mm.step(4)
    assert mm.m.DT == 5 and mm.m.ST == 5 and mm.m.V[1] == 6


def test_key_skips(oracle_lib):
    for op, key, v, skip in ((0xE09E, 7, 7, True), (0xE09E, 3, 7, False), (0xE09E, -1, 7, False),
                             (0xE0A1, 7, 7, False), (0xE0A1, 3, 7, True), (0xE0A1, -1, 7, True),
                             (0xE09E, 7, 0x17, True)):
        m = machine(oracle_lib, [op])
        m.set_V(0, v)
        m.exec(key=key)
        assert m.m.PC == (0x204 if skip else 0x202)


def test_wait_for_key(oracle_lib):
    m = machine(oracle_lib, [0xF30A, 0x1202])
    m.exec(5)
    assert m.m.PC == 0x200 and m.m.V[3] == 0
    m.exec(key=9)
    assert m.m.PC == 0x202 and m.m.V[3] == 9


# ---------------------------------------------------------------- environment wrapper
# V6 += 1 once per frame, synchronised by a 1-frame delay-timer wait.
RAMP = [0x7601, 0x6401, 0xF415, 0xF407, 0x3400, 0x1206, 0x1200]


def test_env_ramp_closed_form(oracle_lib):
    """Score +1 per frame, frame skip 4 -> reward 4 per step; done when
    V6 >= 20 (after 20 frames = 5 steps); auto-reset restarts the episode."""
    g = prog(RAMP, instr_per_frame=10, frameskip=4, score=(Term("reg", 6),),
             term=(Clause(Term("reg", 6), ">=", 20),))
    e = oracle_lib.OracleEnv([g], 3, seed=5)
    obs0 = e.reset()
    assert np.all(obs0 == 0)
    rewards, dones = [], []
    for t in range(12):
        o, r, d = e.step(np.array([0, 1, 4], dtype=np.uint8))
        rewards.append(r.copy())
        dones.append(d.copy())
    R = np.array(rewards)
    D = np.array(dones)
    assert np.all(R[:, 0] == [4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4])
    assert list(np.nonzero(D[:, 0])[0]) == [4, 9]
    assert np.all(R == R[:, :1]) and np.all(D == D[:, :1])
    rec = e.records()
    assert np.all(rec["episode_steps"] == 2) and np.all(rec["env_steps"] == 12)


def test_env_truncation_and_actions(oracle_lib):
    g = prog(RAMP, instr_per_frame=10, frameskip=4, score=(Term("reg", 6),),
             max_episode_steps=3, action_set=(1, 2))
    e = oracle_lib.OracleEnv([g], 3)
    e.reset()
    d_hist = []
    for t in range(7):
        _, r, d = e.step(np.array([0, 2, 3], dtype=np.uint8))
        d_hist.append(int(d[0]))
    assert d_hist == [0, 0, 1, 0, 0, 1, 0]
    st = e.records()["status"]
    assert list(st) == [0, 0, oracle_lib.ST_BAD_ACTION]


def test_instructions_per_frame(oracle_lib):
    for k, fs in ((10, 4), (5, 4), (20, 2), (7, 3)):
        g = prog([0x7001, 0x1200], instr_per_frame=k, frameskip=fs, stack_frames=1)
        m = oracle_lib.Machine(g)
        m.step(0)
        assert m.m.V[0] == (k * fs + 1) // 2


def test_observation_frames(oracle_lib):
    """The observation stacks the last frames of the step, oldest first, and
    each is the display at the end of its frame (§3.2)."""
    # one pixel moves right by one column per frame
    words = [0xA20E, 0x6001, 0xD011, 0xF015, 0xF107, 0x3100, 0x1208, 0xD011, 0x7001,
             0xD011, 0x6101, 0xF115, 0x1208, 0x8000]
    data = bytes([0x80])
    for fs, S in ((4, 4), (4, 2), (3, 1)):
        g = prog(words, data, instr_per_frame=10, frameskip=fs, stack_frames=S)
        m = oracle_lib.Machine(g)
        ref = oracle_lib.Machine(g)
        frames = []
        for f in range(fs):
            ref.exec(10)
            ref.tick()
            frames.append(ref.pixels)
        o, _, _ = m.step(0)
        assert o.shape == (S, 32, 64)
        for s in range(S):
            assert np.array_equal(o[s], frames[fs - S + s])
        assert np.array_equal(o[-1], m.pixels)
        assert set(np.unique(o)) <= {0, 1}


def test_startup_instructions(oracle_lib):
    """§3.3 "Initialization handling": startup instructions run at reset."""
    g = prog([0x7001, 0x1200], startup_instrs=25, instr_per_frame=10)
    m = oracle_lib.Machine(g)
    assert m.m.V[0] == 13 and m.m.PC == 0x202
    g2 = prog([0x6007, 0xF015, 0x1204], startup_instrs=23, instr_per_frame=10)
    m2 = oracle_lib.Machine(g2)
    assert m2.m.DT == 5  # ticked after instructions 10 and 20


# ---------------------------------------------------------------- reward/termination
@pytest.mark.parametrize("name", sorted(PAPER_GAMES))
def test_paper_score_and_termination_expressions(oracle_lib, name):
    score, term = PAPER_GAMES[name]
    g = GameSpec(rom=b"\x12\x00", score=score, term=term)
    m = oracle_lib.Machine(g)
    s_fn, t_fn = PAPER_EXPR[name]
    rng = np.random.default_rng(hash(name) % 2**32)
    regs = {t.lhs.idx for t in term} | {t.idx for t in score}
    for r in regs:
        for v in range(256):
            V = [int(x) for x in rng.integers(0, 256, 16)]
            V[r] = v
            for i in range(16):
                m.set_V(i, V[i])
            assert m.score() == s_fn(V), (name, r, v)
            assert m.terminated() == bool(t_fn(V)), (name, r, v)


def test_bcd_nibble_score_reading(oracle_lib):
    """App. E reading of Pong: 0x23 means player 2, opponent 3."""
    g = GameSpec(rom=b"\x12\x00", score=(Term("reg", 14, "nib_hi_minus_lo"),))
    m = oracle_lib.Machine(g)
    m.set_V(14, 0x23)
    assert m.score() == -1
    m.set_V(14, 0x90)
    assert m.score() == 9


def test_memory_score_term(oracle_lib):
    g = GameSpec(rom=bytes([0xA3, 0x00, 0xF3, 0x33, 0x12, 0x04]),
                 score=(Term("mem", 0x301, "raw"), Term("mem", 0x302, "neg")))
    m = oracle_lib.Machine(g)
    m.set_V(3, 147)
    m.exec(2)
    assert m.score() == 4 - 7


# ---------------------------------------------------------------- randomness
def test_rnd_masks_and_determinism(oracle_lib):
    m = machine(oracle_lib, [0xC000, 0x1200], seed=9)
    for _ in range(20):
        m.exec(2)
        assert m.m.V[0] == 0
    vals = []
    m = machine(oracle_lib, [0xC0FF, 0x8104, 0xC00F, 0x1200], seed=9)
    for _ in range(4000):
        m.exec()
        if m.m.PC == 0x202:
            vals.append(m.m.V[0])
    vals = np.array(vals)
    counts = np.bincount(vals, minlength=256)
    # chi-square against uniform bytes (255 dof): far inside the 1e-6 tail
    exp = len(vals) / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 400


def test_rnd_streams_depend_on_identity_not_batch(oracle_lib):
    """Counter-based draws: an instance's trajectory depends on (seed, uid,
    step), not on which other instances share the batch."""
    from paper_2510_01764_gb300.workloads import actions, random_game
    g = random_game(7)
    n = 16
    acts = actions(11, 0, 30, n)
    e1 = oracle_lib.OracleEnv([g], n, seed=3)
    _, r1, d1, h1 = e1.rollout(acts, hashes=True)
    perm = np.random.default_rng(0).permutation(n)
    e2 = oracle_lib.OracleEnv([g], n, seed=3, uid_of_env=perm)
    _, r2, d2, h2 = e2.rollout(acts[:, perm], hashes=True)
    assert np.array_equal(h2, h1[:, perm])
    e3 = oracle_lib.OracleEnv([g], n, seed=4)
    _, _, _, h3 = e3.rollout(acts, hashes=True)
    assert not np.array_equal(h3[-1], h1[-1])
    assert len(set(h1[-1].tolist())) > n // 2  # most uids diverge


# ---------------------------------------------------------------- quirks
def test_quirk_bits_change_only_their_opcode(oracle_lib):
    m = machine(oracle_lib, [0x8016], quirks=0x01)
    m.set_V(0, 0xF0); m.set_V(1, 0x03)
    m.exec()
    assert m.m.V[0] == 0x01 and m.m.V[15] == 1
    m = machine(oracle_lib, [0xA300, 0xF255], quirks=0x02)
    m.exec(2)
    assert m.m.I == 0x303
    m = machine(oracle_lib, [0x8011], quirks=0x04)
    m.m.V[15] = 5
    m.exec()
    assert m.m.V[15] == 0
    m = machine(oracle_lib, [0xB310], quirks=0x08)
    m.set_V(3, 2); m.set_V(0, 100)
    m.exec()
    assert m.m.PC == 0x312


def test_state_hash_is_fnv_of_record(oracle_lib):
    from paper_2510_01764_gb300.workloads import actions, cfg_small
    w = cfg_small()
    e = oracle_lib.OracleEnv(w.games, 4, seed=w.seed)
    e.rollout(actions(1, 0, 50, 4))
    recs = e.records()
    hs = e.hashes()
    for i in range(4):
        assert oracle_lib.fnv1a64(canonical_bytes(recs[i], "chip8")) == int(hs[i])


def canonical_bytes(r, variant: str) -> bytes:
    """The hashed serialisation of a record, field by field, little-endian:
    CHIP-8 hashes display rows 0-31 (word 0); SCHIP all 64 x 2 words, then
    hires and the 16 flag bytes after last_action."""
    head = (r["V"].tobytes() + r["I"].tobytes() + r["PC"].tobytes() +
            bytes([r["SP"], r["DT"], r["ST"], r["status"]]) + r["stack"].tobytes())
    disp = r["display"].tobytes() if variant == "schip" else r["display"][:32, 0].tobytes()
    tail = r["episode_steps"].tobytes() + r["env_steps"].tobytes() + bytes([r["last_action"]])
    if variant == "schip":
        tail += bytes([r["hires"]]) + r["rpl"].tobytes()
    return head + disp + r["ram"].tobytes() + tail


# ---------------------------------------------------------------- wrappers (§3.2)
# Echo program: every frame V3 = 1..4 for held key 7/9/5/8 (EXA1 skips the
# assignment when the key is up), 0 for none; then wait for the delay timer so
# that one pass runs per frame.
ECHO = [
    0x6300,                   # 0x200 V3 = 0 (no key)
    0x6507, 0xE5A1, 0x6301,   # 0x202 key 7 held -> V3 = 1
    0x6509, 0xE5A1, 0x6302,   # key 9 -> 2
    0x6505, 0xE5A1, 0x6303,   # key 5 -> 3
    0x6508, 0xE5A1, 0x6304,   # key 8 -> 4
    0x6401, 0xF415,           # 0x21A DT = 1
    0xF407, 0x3400, 0x121E,   # 0x21E wait for DT == 0
    0x1200,
]


def _echo(**kw):
    g = prog(ECHO, instr_per_frame=40, frameskip=1, stack_frames=1, **kw)
    return g


def test_sticky_off_matches_agent_actions(oracle_lib):
    g = _echo()
    m = oracle_lib.Machine(g)
    acts = [0, 1, 2, 3, 4, 2, 0]
    for a in acts:
        m.step(a)
        assert m.m.V[3] == (0 if a == 4 else a + 1)
        assert m.m.last_action == a


def test_sticky_always_repeats_previous_action(oracle_lib):
    """p -> 1: every step repeats the previous action, which at episode start
    is the no-op, so the agent's keys never reach the program."""
    g = _echo(sticky_prob=1.0 - 2.0 ** -33)
    m = oracle_lib.Machine(g)
    for a in (0, 1, 2, 3, 0, 1):
        m.step(a)
        assert m.m.V[3] == 0 and m.m.last_action == 4


def test_sticky_frequency(oracle_lib):
    """p = 0.25: about a quarter of the steps apply the previous action."""
    g = _echo(sticky_prob=0.25)
    rng = np.random.default_rng(0)
    repeats, changes = 0, 0
    for uid in range(40):
        m = oracle_lib.Machine(g, seed=3, uid=uid)
        prev = 4
        for t in range(50):
            a = int(rng.integers(0, 4))
            m.step(a)
            applied = m.m.last_action
            assert applied in (a, prev)
            if a != prev:
                changes += 1
                repeats += applied == prev
            prev = applied
    frac = repeats / changes
    assert 0.20 < frac < 0.30, frac


def test_noop_reset_counts(oracle_lib):
    """No-op reset: 0..max no-key steps (frameskip frames each) before the
    episode starts; every count occurs and the episode step count is 0."""
    g = prog([0x7001, 0x6401, 0xF415, 0xF407, 0x3400, 0x1206, 0x1200],  # V0 += 1 per frame
             instr_per_frame=10, frameskip=4, stack_frames=1, max_noops=5)
    seen = set()
    for uid in range(300):
        m = oracle_lib.Machine(g, seed=11, uid=uid)
        frames = m.m.V[0]
        # one increment per frame; n no-op steps = 4n frames
        assert frames % 4 == 0, frames
        seen.add(frames)
        assert m.m.episode_steps == 0 and m.m.last_action == len(g.action_set)
    assert seen == {4 * k for k in range(6)}


def _chi2_uniform(counts) -> float:
    counts = np.asarray(counts, dtype=np.float64)
    e = counts.sum() / len(counts)
    return float(((counts - e) ** 2 / e).sum())


def test_rnd_bytes_are_uniform(oracle_lib):
    """CXNN with NN = FF over 40,000 draws (many instances and steps): the
    byte histogram passes a chi-square test (255 dof; 99.9 % point ~ 330)."""
    g = prog([0xC0FF, 0x8104, 0x1200], instr_per_frame=3, frameskip=1, stack_frames=1)  # one draw a step
    e = oracle_lib.OracleEnv([g], 400, seed=77)
    e.reset()
    seen = []
    for _ in range(100):
        e.step(np.zeros(400, np.uint8))
        seen.append(e.records()["V"][:, 0].copy())
    counts = np.bincount(np.concatenate(seen), minlength=256)
    assert _chi2_uniform(counts) < 330, counts


def test_noop_count_is_uniform(oracle_lib):
    """No-op reset with max 7: the number of no-op frames over 4,000
    identities is uniform over 0..7 (7 dof; 99.9 % point ~ 24.3)."""
    g = prog([0x7001, 0x6401, 0xF415, 0xF407, 0x3400, 0x1206, 0x1200],
             instr_per_frame=10, frameskip=1, stack_frames=1, max_noops=7)
    e = oracle_lib.OracleEnv([g], 4000, seed=5)
    counts = np.bincount(e.records()["V"][:, 0], minlength=8)
    assert counts.sum() == 4000 and len(counts) == 8
    assert _chi2_uniform(counts) < 24.3, counts


# ---------------------------------------------------------------- code as data
# An instruction rewritten by FX55 runs as its new bytes; a jump to an odd
# address fetches the opcode that straddles the word boundary (§3.2: the
# opcode is the two bytes at PC, whatever PC is).
PATCH = [0x6A05,  # 0x200 VA = 5        (rewritten below to 6A09: VA = 9)
         0x7B01,  # 0x202 VB += 1
         0x3B02,  # 0x204 skip next if VB == 2
         0x120A,  # 0x206 first pass: go and patch
         0x1208,  # 0x208 second pass: park here
         0x606A,  # 0x20A V0 = 0x6A
         0x6109,  # 0x20C V1 = 0x09
         0xA200,  # 0x20E I = 0x200
         0xF155,  # 0x210 RAM[0x200..0x201] = V0, V1
         0x1200]  # 0x212 back to the rewritten instruction
ODD = bytes([0x12, 0x03,         # 0x200 jump 0x203
             0x00, 0x6C, 0x07,   # 0x203: 6C07 (VC = 7)
             0x12, 0x05])        # 0x205: 1205 (park at an odd address)


def test_rewritten_instruction_runs_as_its_new_bytes(oracle_lib):
    m = machine(oracle_lib, PATCH)
    m.exec(12)                     # 4 + 5 (patch) + 3 instructions
    assert m.V[10] == 9 and m.V[11] == 2 and m.m.PC == 0x208
    assert list(m.ram[0x200:0x202]) == [0x6A, 0x09]
    m.exec(5)
    assert m.m.PC == 0x208 and m.V[10] == 9


def test_odd_pc_fetches_the_straddling_opcode(oracle_lib):
    from chip8_prog import GameSpec
    m = oracle_lib.Machine(GameSpec(rom=ODD, action_set=(7, 9, 5, 8)))
    m.exec(2)
    assert m.V[12] == 7 and m.m.PC == 0x205
    m.exec(3)
    assert m.m.PC == 0x205 and m.m.status == 0


# Sprites on a page that the program writes (§3.2 memory, App. B DXYN): the
# drawn rows are the RAM's current bytes, whether or not they were written.
SPRITE_PAGE_WORDS = [0xA230,  # I = 0x230 (score buffer, same 64-byte page as the sprites)
                     0x6A7B,  # VA = 123
                     0xFA33,  # BCD into 0x230-0x232
                     0xA228,  # I = sprite A (0x228-0x22C)
                     0x6305, 0x6404,
                     0xD345,  # draw A at (5, 4)
                     0x60FF, 0x6181,
                     0xA229,
                     0xF155,  # rewrite A's rows 1-2 with FF 81
                     0xA228, 0x6414,
                     0xD345,  # draw A again at (5, 20)
                     0xA22D, 0x631E,
                     0xD343,  # draw B (0x22D-0x22F, unchanged) at (30, 20)
                     0x1222, 0x0000, 0x0000]
SPRITE_PAGE_DATA = bytes([0xF0, 0x90, 0xF0, 0x90, 0xF0,  # A at 0x228
                          0x3C, 0x66, 0x3C,              # B at 0x22D
                          0, 0, 0, 0])                   # score buffer at 0x230


def test_sprites_on_a_written_page(oracle_lib):
    m = machine(oracle_lib, SPRITE_PAGE_WORDS, data=SPRITE_PAGE_DATA)
    m.exec(18)
    assert m.m.PC == 0x222
    assert list(m.ram[0x230:0x233]) == [1, 2, 3]

    def rows(y, x, n):
        return [int("".join(str(int(b)) for b in m.pixels[y + r, x:x + 8]), 2) for r in range(n)]

    assert rows(4, 5, 5) == [0xF0, 0x90, 0xF0, 0x90, 0xF0]
    assert rows(20, 5, 5) == [0xF0, 0xFF, 0x81, 0x90, 0xF0]
    assert rows(20, 30, 3) == [0x3C, 0x66, 0x3C]
    assert m.pixels.sum() == sum(bin(v).count("1") for v in (0xF0, 0x90) * 2 + (0xF0,)) \
        + sum(bin(v).count("1") for v in (0xF0, 0xFF, 0x81, 0x90, 0xF0, 0x3C, 0x66, 0x3C))


def test_oracle_command_line(oracle_lib, tmp_path):
    """`python -m oracle` prints the same per-step hashes as the library."""
    import subprocess
    import sys

    from paper_2510_01764_gb300 import workloads as W

    rom = W.template_rom(W.TemplateParams(seed=3))
    path = tmp_path / "t.ch8"
    path.write_bytes(rom)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-m", "oracle", str(path), "--envs", "3", "--steps", "5"],
                         capture_output=True, text=True, check=True, cwd=root).stdout.splitlines()
    game = W.GameSpec(rom=rom, action_set=(7, 9, 5, 8), score=(W.Term("reg", 6),))
    env = oracle_lib.OracleEnv([game], 3, seed=1)
    env.reset()
    _, r, d, h = env.rollout(W.actions(1, 0, 5, 3, 5), hashes=True)
    for s in range(5):
        assert out[s].split() == [str(s)] + [f"{int(x):016x}" for x in h[s]]
    assert out[5].split() == ["reward", f"{float(r.sum()):.0f}", "done", str(int(d.sum()))]


# ---------------------------------------------------------------- DXYN brute force
def _dxyn_by_planes(bg, rows, x0, y0, wrap):
    """App. B sprite drawing restated as plane arithmetic: the sprite's bits
    (MSB leftmost) placed on a padded plane at (x0, y0), the overhang either
    dropped (clip) or folded back onto the opposite edge (wrap); the display
    becomes bg XOR plane and VF says whether the plane met a lit pixel."""
    n = len(rows)
    plane = np.zeros((32 + 16, 64 + 8), dtype=np.uint8)
    if n:
        bits = np.unpackbits(np.frombuffer(bytes(rows), dtype=np.uint8)).reshape(n, 8)
        plane[y0:y0 + n, x0:x0 + 8] = bits
    on = plane[:32, :64].copy()
    if wrap:
        on[:16, :] |= plane[32:, :64]
        on[:, :8] |= plane[:32, 64:]
        on[:16, :8] |= plane[32:, 64:]
    return bg ^ on, int((bg & on).any())


@pytest.mark.parametrize("wrap", [False, True])
@pytest.mark.parametrize("pattern", ["full", "random", "sparse"])
def test_dxyn_brute_force_every_position_and_height(oracle_lib, pattern, wrap):
    """Every origin (x0, y0) of the 64x32 display and every height N = 0..15
    (VX, VY also above 63 / 31, reduced mod 64 / 32), over backgrounds that
    are empty, sparse, dense or a checkerboard, with and without the
    sprite-wrap quirk: the oracle's display and VF equal the plane
    definition above."""
    rng = np.random.default_rng({"full": 1, "random": 2, "sparse": 3}[pattern])
    sprite = {"full": bytes([0xFF] * 15),
              "random": bytes(rng.integers(0, 256, 15, dtype=np.uint8)),
              "sparse": bytes([0x81, 0x00, 0x18, 0x24, 0x00, 0x42, 0x80, 0x01, 0x00,
                               0x10, 0x08, 0x00, 0xC0, 0x03, 0x66])}[pattern]
    checker = (np.indices((32, 64)).sum(axis=0) % 2).astype(np.uint8)
    bgs = [np.zeros((32, 64), np.uint8), (rng.random((32, 64)) < 0.05).astype(np.uint8),
           (rng.random((32, 64)) < 0.5).astype(np.uint8), checker]
    code = [0xD010 | n for n in range(16)]
    m = machine(oracle_lib, code, data=sprite, quirks=0x10 if wrap else 0)
    ram = np.ctypeslib.as_array(m.m.ram)
    i_sprite = int(np.nonzero([bytes(ram[a:a + 15]) == sprite for a in range(0x200, 0x240)])[0][0]) + 0x200
    pix = np.ctypeslib.as_array(m.m.pix)
    hits = 0
    for n in range(16):
        for y0 in range(32):
            for x0 in range(64):
                bg = bgs[(x0 + 3 * y0 + n) % 4]
                pix[:] = 0
                pix[:32, :64] = bg
                m.m.PC = 0x200 + 2 * n
                m.m.I = i_sprite
                m.m.V[0] = x0 + 64 * ((y0 + n) % 4)
                m.m.V[1] = y0 + 32 * (x0 % 8)
                m.m.V[15] = 7
                m.exec()
                want, vf = _dxyn_by_planes(bg, sprite[:n], x0, y0, wrap)
                assert np.array_equal(pix[:32, :64], want), (x0, y0, n)
                assert m.m.V[15] == vf, (x0, y0, n)
                assert not pix[32:].any() and not pix[:, 64:].any()
                hits += vf
    assert hits > 1000


def test_dxyn_sprite_rows_wrap_around_memory(oracle_lib):
    """Sprite rows are read at (I + r) mod 4096: a 15-row sprite starting at
    0xFF8 takes its last 7 rows from 0x000-0x006."""
    sprite = bytes(range(0x11, 0x11 + 15 * 0x0B, 0x0B))
    m = machine(oracle_lib, [0xD01F])
    ram = np.ctypeslib.as_array(m.m.ram)
    ram[0xFF8:0x1000] = np.frombuffer(sprite[:8], np.uint8)
    ram[0x000:0x007] = np.frombuffer(sprite[8:], np.uint8)
    m.m.I = 0xFF8
    m.m.V[0], m.m.V[1] = 20, 9
    m.exec()
    want, vf = _dxyn_by_planes(np.zeros((32, 64), np.uint8), sprite, 20, 9, False)
    assert np.array_equal(m.pixels, want) and m.m.V[15] == vf == 0
