"""Pins of the oracle's Super-CHIP variant (the 128x64 extension that §5 of the
paper names) to facts outside its own code: the CHIP-8 semantics already
pinned (a lores SCHIP run of a CHIP-8 program must reproduce the CHIP-8
screen with every pixel drawn as a 2x2 block), sprite placement computed
with numpy, scrolls as numpy shifts with zero fill, and the instruction
definitions (modes, exit, flag registers, big-glyph addresses).
"""
import numpy as np
import pytest

from chip8_prog import prog
from paper_2510_01764_gb300 import workloads as W
from paper_2510_01764_gb300.workloads import GameSpec
from test_oracle_pins import canonical_bytes


def schip(oracle, words, data=b"", **kw):
    kw.setdefault("variant", "schip")
    return oracle.Machine(prog(words, data, **kw))


def place(sprite_rows, width, x0, y0, W_, H_):
    """Expected buffer after XOR-drawing a sprite on an empty W_ x H_ grid
    (clipping at the right and bottom edges)."""
    g = np.zeros((H_, W_), dtype=np.uint8)
    for r, bits in enumerate(sprite_rows):
        for c in range(width):
            if (bits >> (width - 1 - c)) & 1 and y0 + r < H_ and x0 + c < W_:
                g[y0 + r, x0 + c] ^= 1
    return g


def test_lores_run_is_chip8_run_doubled(oracle_lib):
    """Template programs (DXYN, FX29, FX33, CXNN, keys, timers) run in SCHIP
    lores mode: registers, RAM outside the big glyphs and the screen match
    the CHIP-8 run, the screen as 2x2 blocks."""
    for seed in (1, 2, 3):
        tp = W.TemplateParams(seed=seed, deco_pairs=2)
        g8 = W.template_game(tp)
        gs = W.replace(g8, variant="schip")
        m8 = oracle_lib.Machine(g8, seed=5, uid=seed)
        ms = oracle_lib.Machine(gs, seed=5, uid=seed)
        rng = np.random.default_rng(seed)
        for step in range(120):
            a = int(rng.integers(0, 5))
            m8.step(a)
            ms.step(a)
            assert m8.V == ms.V and m8.m.PC == ms.m.PC and m8.m.I == ms.m.I
            assert np.array_equal(np.kron(m8.pixels, np.ones((2, 2), np.uint8)), ms.pixels)
        r8, rs = m8.ram, ms.ram
        assert np.array_equal(r8[:0xA0], rs[:0xA0]) and np.array_equal(r8[0x140:], rs[0x140:])


def test_hires_dxyn_placement_and_clipping(oracle_lib):
    rng = np.random.default_rng(0)
    sprite = bytes(int(b) for b in rng.integers(1, 256, 15))
    # 0x200: hires; V0 = x, V1 = y preset by the test; I = sprite; D01N
    for n in (1, 5, 15):
        for x, y in [(0, 0), (120, 0), (127, 63), (60, 59), (121, 50), (64, 32), (3, 63)]:
            m = schip(oracle_lib, [0x00FF, 0xA208, 0xD010 | n, 0x1206], data=sprite)
            m.exec()                       # hires
            m.set_V(0, x)
            m.set_V(1, y)
            m.exec(2)
            exp = place(sprite[:n], 8, x, y, 128, 64)
            assert np.array_equal(m.pixels, exp), (n, x, y)
            assert m.V[15] == 0
            m.m.PC = 0x202
            m.exec(2)                      # draw again: erased, collision
            assert not m.pixels.any() and m.V[15] == int(exp.any())


def test_coordinates_wrap_modulo_the_grid(oracle_lib):
    """VX mod 128 / VY mod 64 in hires, mod 64 / 32 in lores."""
    m = schip(oracle_lib, [0x00FF, 0xA206, 0xD011], data=bytes([0x80]))
    m.exec()
    m.set_V(0, 130)
    m.set_V(1, 70)
    m.exec(2)
    assert m.pixels[6, 2] == 1 and m.pixels.sum() == 1
    m = schip(oracle_lib, [0xA204, 0xD011], data=bytes([0x80]))
    m.set_V(0, 70)
    m.set_V(1, 35)
    m.exec(2)
    assert m.pixels[6:8, 12:14].all() and m.pixels.sum() == 4


@pytest.mark.parametrize("hires", [0, 1])
def test_dxy0_draws_16x16(oracle_lib, hires):
    rng = np.random.default_rng(hires)
    big = bytes(int(b) for b in rng.integers(0, 256, 32))
    rows = [big[2 * r] << 8 | big[2 * r + 1] for r in range(16)]
    for x, y in [(0, 0), (10, 7), (120, 60), (56, 28)]:
        pre = [0x00FF] if hires else [0x00FE]
        m = schip(oracle_lib, pre + [0xA208, 0xD010, 0x1206], data=big)
        m.exec()
        m.set_V(0, x)
        m.set_V(1, y)
        m.exec(2)
        if hires:
            exp = place(rows, 16, x % 128, y % 64, 128, 64)
        else:
            exp = np.kron(place(rows, 16, x % 64, y % 32, 64, 32), np.ones((2, 2), np.uint8))
        assert np.array_equal(m.pixels, exp), (hires, x, y)


def _random_buffer(m, seed):
    rng = np.random.default_rng(seed)
    buf = rng.integers(0, 2, (64, 128)).astype(np.uint8)
    for y in range(64):
        for x in range(128):
            m.m.pix[y][x] = int(buf[y, x])
    return buf


@pytest.mark.parametrize("hires", [0, 1])
def test_scrolls_are_shifts_with_zero_fill(oracle_lib, hires):
    unit = 1 if hires else 2
    for op in [0x00C1, 0x00C4, 0x00CF, 0x00FB, 0x00FC, 0x00C0]:
        m = schip(oracle_lib, [0x00FF if hires else 0x00FE, op])
        m.exec()
        buf = _random_buffer(m, op)
        m.exec()
        exp = np.zeros_like(buf)
        if (op & 0xFFF0) == 0x00C0:
            k = (op & 15) * unit
            exp[k:] = buf[:64 - k] if k else buf
        elif op == 0x00FB:
            exp[:, 4 * unit:] = buf[:, :128 - 4 * unit]
        else:
            exp[:, :128 - 4 * unit] = buf[:, 4 * unit:]
        assert np.array_equal(m.pixels, exp), hex(op)


def test_mode_switch_keeps_the_buffer(oracle_lib):
    glyph = bytes([0xF0, 0x90, 0xF0, 0x90, 0xF0])
    m = schip(oracle_lib, [0xA208, 0xD015, 0x00FF, 0x00FE], data=glyph)
    m.exec(2)
    before = m.pixels
    exp = np.kron(place(glyph, 8, 0, 0, 64, 32), np.ones((2, 2), np.uint8))
    assert m.m.hires == 0 and np.array_equal(before, exp)
    m.exec()
    assert m.m.hires == 1 and np.array_equal(m.pixels, before)
    m.exec()
    assert m.m.hires == 0 and np.array_equal(m.pixels, before)


def test_exit_halts_with_status(oracle_lib):
    m = schip(oracle_lib, [0x6001, 0x00FD, 0x6002])
    m.exec(10)
    assert m.m.PC == 0x202 and m.V[0] == 1
    assert m.m.status & oracle_lib.ST_EXIT


def test_flag_registers_roundtrip(oracle_lib):
    for x in range(16):
        m = schip(oracle_lib, [0xF075 | x << 8, 0x6000, 0x6100, 0x6F00, 0xF085 | x << 8])
        for i in range(16):
            m.set_V(i, 10 + i)
        m.exec()
        assert list(m.m.rpl)[:x + 1] == [10 + i for i in range(x + 1)]
        assert all(v == 0 for v in list(m.m.rpl)[x + 1:])
        m.exec(4)
        expect = [10 + i for i in range(x + 1)] + [10 + i for i in range(x + 1, 16)]
        expect = [expect[i] if i <= x else (0 if i in (0, 1, 15) else 10 + i) for i in range(16)]
        assert m.V == expect


def test_big_glyph_addresses(oracle_lib):
    for v in range(256):
        m = schip(oracle_lib, [0xF330])
        m.set_V(3, v)
        m.exec()
        assert m.m.I == 0xA0 + 10 * (v % 16)
    ram = schip(oracle_lib, [0x1200]).ram
    glyphs = ram[0xA0:0x140].reshape(16, 10)
    assert all(g.any() for g in glyphs) and len({bytes(g) for g in glyphs}) == 16
    assert np.all(ram[0x140:0x200] == 0)


def test_schip_opcodes_in_chip8_mode(oracle_lib):
    """In the CHIP-8 variant the SCHIP 00xx forms are ignored machine-code
    calls and FX30/75/85 are undefined."""
    m = oracle_lib.Machine(prog([0xA20C, 0xD015, 0x00FF, 0x00C3, 0x00FB, 0x00FD],
                                data=bytes([0xF0] * 5)))
    m.exec(2)
    before = m.pixels
    m.exec(4)
    assert np.array_equal(m.pixels, before) and m.m.PC == 0x20C and m.m.status == 0
    for op in (0xF030, 0xF075, 0xF085):
        m = oracle_lib.Machine(prog([op]))
        m.exec()
        assert m.m.status & oracle_lib.ST_BAD_OP


def test_reset_restores_lores_and_clears_flags(oracle_lib):
    g = prog([0x00FF, 0x6007, 0xF075, 0x1206], variant="schip", startup_instrs=3)
    m = oracle_lib.Machine(g)
    assert m.m.hires == 1 and m.m.rpl[0] == 7
    e = oracle_lib.OracleEnv([prog([0x00FF, 0x6007, 0xF075, 0x1206], variant="schip",
                                   max_episode_steps=1)], 2)
    e.reset()
    e.step(np.zeros(2, np.uint8))
    rec = e.records()
    assert (rec["hires"] == 0).all() and (rec["rpl"] == 0).all()


def test_observations_and_hash(oracle_lib):
    g = W.replace(W.template_game(W.TemplateParams(seed=4)), variant="schip")
    e = oracle_lib.OracleEnv([g], 6, seed=2)
    obs0 = e.reset()
    assert obs0.shape == (6, 4, 64, 128)
    o, r, d = e.step(np.array([0, 1, 2, 3, 4, 0], np.uint8))
    recs = e.records()
    for i in range(6):
        bits = np.unpackbits(recs[i]["display"].view(np.uint8).reshape(64, 16), axis=1,
                             bitorder="little")
        assert np.array_equal(bits, o[i, -1])
    hs = e.hashes()
    for i in range(6):
        assert oracle_lib.fnv1a64(canonical_bytes(recs[i], "schip")) == int(hs[i])


def test_variant_is_per_environment(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.OracleEnv([GameSpec(rom=b"\x12\x00"), GameSpec(rom=b"\x12\x00", variant="schip")], 2,
                             game_of_env=np.array([0, 1], np.uint16))
