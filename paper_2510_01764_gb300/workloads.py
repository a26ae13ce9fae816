"""Seeded synthetic inputs for the vectorised CHIP-8 environment step.

This module writes inputs only: CHIP-8 machine code (ROM images), game
descriptors (reward / termination registers, action sets) and action streams.
It holds none of the emulator's arithmetic; the CUDA path and the CPU oracle
both consume what it produces, and it imports neither of them.

The paper's workloads are third-party game ROMs (§3.4, App. C) that are not
available here. The generators below stand in for them with programs shaped
like the arcade games the paper describes (§3.2-§3.3): key polls with
EX9E/EXA1 over a 4-key action set, sprites moved by erase/redraw DXYN pairs,
collision detection through VF, a score register drawn with FX33/FX65/FX29,
delay-timer waits with FX15/FX07 and random spawn positions with CXNN.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Sequence

import numpy as np

# --------------------------------------------------------------------------
# Game descriptor (§3.3: score_fn, terminated_fn, action_set,
# startup_instructions; §3.2: frame skip, 4-frame stack).


@dataclass(frozen=True)
class Term:
    """One score / termination term: a register or memory byte, transformed.

    src: "reg" (V[idx]) or "mem" (RAM[idx]).
    xform: "raw", "neg", "dec_tens", "dec_ones", "dec_tens_minus_ones",
           "nib_hi_minus_lo", "zero_if_gt" (arg = threshold).
    """

    src: str
    idx: int
    xform: str = "raw"
    arg: int = 0


@dataclass(frozen=True)
class Clause:
    """Termination clause: ``lhs <cmp> rhs`` with cmp in == != >= > <= <."""

    lhs: Term
    cmp: str
    rhs: int


@dataclass(frozen=True)
class GameSpec:
    rom: bytes
    instr_per_frame: int = 10
    frameskip: int = 4
    stack_frames: int = 4
    action_set: tuple = (7, 9, 5, 8)
    score: tuple = ()          # Terms, summed
    term: tuple = ()           # Clauses, OR-ed; empty = never terminates
    max_episode_steps: int = 0  # 0 = no truncation
    startup_instrs: int = 0
    sticky_prob: float = 0.0    # sticky actions: repeat the previous action w.p. this
    max_noops: int = 0          # no-op reset: 0..max_noops no-key steps per reset
    variant: str = "chip8"      # "chip8" (64x32 screen) or "schip" (128x64 buffer, Super-CHIP)
    name: str = ""

    @property
    def n_actions(self) -> int:
        return len(self.action_set)


XFORMS = ("raw", "neg", "dec_tens", "dec_ones", "dec_tens_minus_ones",
          "nib_hi_minus_lo", "zero_if_gt")
CMPS = ("==", "!=", ">=", ">", "<=", "<")


# --------------------------------------------------------------------------
# A tiny two-pass CHIP-8 assembler: emits big-endian opcode words, resolves
# label references for jumps, calls and I loads.


class Asm:
    def __init__(self, origin: int = 0x200):
        self.origin = origin
        self.buf = bytearray()
        self.labels: dict[str, int] = {}
        self.fixups: list[tuple[int, int, str]] = []  # (offset, high nibble, label)

    @property
    def here(self) -> int:
        return self.origin + len(self.buf)

    def label(self, name: str) -> None:
        assert name not in self.labels, name
        self.labels[name] = self.here

    def op(self, word: int) -> None:
        assert 0 <= word <= 0xFFFF
        self.buf += bytes(((word >> 8) & 0xFF, word & 0xFF))

    def ref(self, high: int, label: str) -> None:
        """Emit ``high << 12 | address(label)`` (1NNN, 2NNN, ANNN, BNNN)."""
        self.fixups.append((len(self.buf), high, label))
        self.buf += b"\x00\x00"

    def data(self, bs: Sequence[int]) -> None:
        self.buf += bytes(bs)

    def assemble(self) -> bytes:
        out = bytearray(self.buf)
        for off, high, name in self.fixups:
            addr = self.labels[name]
            assert 0 <= addr <= 0xFFF
            word = (high << 12) | addr
            out[off] = word >> 8
            out[off + 1] = word & 0xFF
        return bytes(out)


# --------------------------------------------------------------------------
# Template arcade ROM.
#
# Registers: V0-V2 BCD digits, V3/V7/VE scratch, V4 delay timer, V5 key,
# V6 score, V8/V9 player x/y, VA/VB object x/y, VC/VD score position, VF flag.

PLAYER_SPRITE = (0x3C, 0x7E, 0xFF, 0x7E, 0x3C)  # 8x5
OBJECT_SPRITE = (0x18, 0x3C, 0x3C, 0x18)        # 8x4
DECO_SPRITE = (0x81, 0x42, 0x24)


@dataclass(frozen=True)
class TemplateParams:
    seed: int
    size: int = 600          # target ROM size in bytes (>= code size)
    alu_ops: int = 8         # seeded ALU/skip filler executed every iteration
    deco_pairs: int = 0      # extra draw+erase DXYN pairs per iteration
    wait_frames: int = 2     # delay-timer wait per iteration
    fall: int = 1            # object fall speed (pixels per iteration)


def template_rom(p: TemplateParams) -> bytes:
    """Seeded arcade-shaped CHIP-8 program (see module docstring)."""
    return _template(p)[0]


def template_labels(p: TemplateParams) -> dict:
    """Addresses of the template's labels (e.g. ``scratch``, the BCD buffer)."""
    return _template(p)[1]


def _template(p: TemplateParams) -> tuple:
    rng = np.random.Generator(np.random.Philox(key=p.seed))
    a = Asm()
    # ---- init
    a.op(0x6800 | 28)          # V8 = player x
    a.op(0x6900 | 26)          # V9 = player y
    a.op(0x6600)               # V6 = score 0
    a.ref(0x2, "draw_score")
    a.op(0x6B00 | 6)           # VB = 6
    a.op(0xCA3F)               # VA = rnd & 63
    a.ref(0xA, "object")
    a.op(0xDAB4)               # draw object
    a.ref(0xA, "player")
    a.op(0xD895)               # draw player
    # ---- main loop
    a.label("loop")
    a.ref(0xA, "player")
    a.op(0xD895)               # erase player
    for key, upd in ((7, 0x78FF), (9, 0x7801), (5, 0x79FF), (8, 0x7901)):
        a.op(0x6500 | key)     # V5 = key
        a.op(0xE5A1)           # skip next if key V5 not held
        a.op(upd)              # move
    a.op(0x6E3F)
    a.op(0x88E2)               # V8 &= 63
    a.op(0x6E1F)
    a.op(0x89E2)               # V9 &= 31
    a.ref(0xA, "player")
    a.op(0xD895)               # redraw player
    # seeded ALU filler on scratch registers (reads game registers only)
    scratch = (0x3, 0x7, 0xE)
    readable = (0x3, 0x7, 0xE, 0x6, 0x8, 0x9, 0xA, 0xB)
    for _ in range(p.alu_ops):
        kind = int(rng.integers(0, 13))
        x = int(scratch[rng.integers(0, 3)])
        y = int(readable[rng.integers(0, len(readable))])
        nn = int(rng.integers(0, 256))
        if kind == 0:
            a.op(0x6000 | x << 8 | nn)
        elif kind == 1:
            a.op(0x7000 | x << 8 | nn)
        elif kind in (2, 3):                     # skip over the next op
            a.op((0x3000 if kind == 2 else 0x4000) | x << 8 | nn)
        else:
            sub = (0x0, 0x1, 0x2, 0x3, 0x4, 0x5, 0x6, 0x7, 0xE)[kind - 4]
            a.op(0x8000 | x << 8 | y << 4 | sub)
    # decorative draw/erase pairs at one seeded spot (raise the DXYN share;
    # each pair leaves the display unchanged)
    if p.deco_pairs:
        a.ref(0xA, "deco")
        a.op(0x6300 | int(rng.integers(0, 56)))   # V3 = x
        a.op(0x6700 | int(rng.integers(8, 24)))   # V7 = y
        for _ in range(p.deco_pairs):
            a.op(0xD373)
            a.op(0xD373)
    # object: erase, fall, respawn at the bottom, redraw, check collision
    a.ref(0xA, "object")
    a.op(0xDAB4)               # erase object
    a.op(0x7B00 | p.fall)      # VB += fall
    a.op(0x6E1B)               # VE = 27
    a.op(0x8EB5)               # VE = 27 - VB, VF = (27 >= VB)
    a.op(0x3F00)               # skip next if VF == 0 (object below 27)
    a.ref(0x1, "no_respawn")
    a.op(0x6B00 | 6)           # VB = 6
    a.op(0xCA3F)               # VA = rnd & 63
    a.label("no_respawn")
    a.ref(0xA, "object")
    a.op(0xDAB4)               # draw object
    a.op(0x3F00)               # skip next if no collision
    a.ref(0x2, "hit")
    # delay wait
    a.op(0x6400 | p.wait_frames)
    a.op(0xF415)               # DT = V4
    a.label("wait")
    a.op(0xF407)               # V4 = DT
    a.op(0x3400)               # skip next if V4 == 0
    a.ref(0x1, "wait")
    a.ref(0x1, "loop")
    # ---- hit: erase object, redraw score + 1, respawn
    a.label("hit")
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.ref(0x2, "draw_score")   # erase old score
    a.op(0x7601)               # score += 1
    a.ref(0x2, "draw_score")   # draw new score
    a.op(0x6B00 | 6)
    a.op(0xCA3F)
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.op(0x00EE)
    # ---- draw_score: 3 BCD digits at (46, 0)
    a.label("draw_score")
    a.ref(0xA, "scratch")
    a.op(0xF633)               # BCD of V6
    a.op(0xF265)               # V0..V2 = digits
    a.op(0x6C00 | 46)
    a.op(0x6D00)
    for d in range(3):
        a.op(0xF029 | d << 8)  # I = glyph(Vd)
        a.op(0xDCD5)
        a.op(0x7C05)
    a.op(0x00EE)
    # ---- data
    a.label("player")
    a.data(PLAYER_SPRITE)
    a.label("object")
    a.data(OBJECT_SPRITE)
    a.label("deco")
    a.data(DECO_SPRITE)
    a.label("scratch")
    a.data((0, 0, 0, 0))
    rom = bytearray(a.assemble())
    if len(rom) < p.size:
        rom += rng.integers(0, 256, size=p.size - len(rom), dtype=np.uint8).tobytes()
    return bytes(rom), dict(a.labels)


def template_game(p: TemplateParams, *, instr_per_frame: int = 10, frameskip: int = 4,
                  score_limit: int = 0, max_episode_steps: int = 0) -> GameSpec:
    """Template ROM + descriptor: reward = V6 increase, done when V6 >= limit."""
    term = (Clause(Term("reg", 6), ">=", score_limit),) if score_limit > 0 else ()
    return GameSpec(rom=template_rom(p), instr_per_frame=instr_per_frame,
                    frameskip=frameskip, stack_frames=4, action_set=(7, 9, 5, 8),
                    score=(Term("reg", 6),), term=term,
                    max_episode_steps=max_episode_steps, startup_instrs=0,
                    name=f"template-{p.seed}")


# --------------------------------------------------------------------------
# Random-opcode ROMs: uniform over the 35 instructions, CXNN at 10 % weight.

OPCODE_KINDS = (
    "0NNN", "00E0", "00EE", "1NNN", "2NNN", "3XNN", "4XNN", "5XY0", "6XNN", "7XNN",
    "8XY0", "8XY1", "8XY2", "8XY3", "8XY4", "8XY5", "8XY6", "8XY7", "8XYE", "9XY0",
    "ANNN", "BNNN", "CXNN", "DXYN", "EX9E", "EXA1", "FX07", "FX0A", "FX15", "FX18",
    "FX1E", "FX29", "FX33", "FX55", "FX65",
)
assert len(OPCODE_KINDS) == 35


def random_opcode_rom(seed: int, n_bytes: int = 3584, cxnn_weight: float = 0.10) -> bytes:
    """``n_bytes // 2`` opcodes drawn from the 35 kinds (CXNN at ``cxnn_weight``,
    the others uniform); jump/call targets even in [0x200, 0xFFE], BNNN bases
    that keep NNN + V0 in range, DXYN heights 1..15."""
    rng = np.random.Generator(np.random.Philox(key=seed + 0x5EED))
    n_ops = n_bytes // 2
    probs = np.full(35, (1.0 - cxnn_weight) / 34.0)
    probs[OPCODE_KINDS.index("CXNN")] = cxnn_weight
    kinds = rng.choice(35, size=n_ops, p=probs)
    xs = rng.integers(0, 16, size=n_ops)
    ys = rng.integers(0, 16, size=n_ops)
    nns = rng.integers(0, 256, size=n_ops)
    nnns = rng.integers(0, 4096, size=n_ops)
    targets = 0x200 + 2 * rng.integers(0, (0xFFE - 0x200) // 2 + 1, size=n_ops)
    bases = rng.integers(0x200, 0xF01, size=n_ops)
    heights = rng.integers(1, 16, size=n_ops)
    out = bytearray()
    for i in range(n_ops):
        k = OPCODE_KINDS[kinds[i]]
        x, y, nn = int(xs[i]), int(ys[i]), int(nns[i])
        if k == "0NNN":
            nnn = int(nnns[i])
            if nnn in (0x0E0, 0x0EE):
                nnn = 0x100
            w = nnn
        elif k == "00E0":
            w = 0x00E0
        elif k == "00EE":
            w = 0x00EE
        elif k in ("1NNN", "2NNN"):
            w = (0x1000 if k == "1NNN" else 0x2000) | int(targets[i])
        elif k == "BNNN":
            w = 0xB000 | int(bases[i])
        elif k == "ANNN":
            w = 0xA000 | int(nnns[i])
        elif k == "DXYN":
            w = 0xD000 | x << 8 | y << 4 | int(heights[i])
        elif k[1:] == "XNN":
            w = int(k[0], 16) << 12 | x << 8 | nn
        elif k[1:3] == "XY":
            w = int(k[0], 16) << 12 | x << 8 | y << 4 | int(k[3], 16)
        else:  # EX9E EXA1 FXnn
            w = int(k[0], 16) << 12 | x << 8 | int(k[2:], 16)
        out += bytes((w >> 8, w & 0xFF))
    return bytes(out)


def random_game(seed: int, *, instr_per_frame: int = 10, frameskip: int = 4) -> GameSpec:
    return GameSpec(rom=random_opcode_rom(seed), instr_per_frame=instr_per_frame,
                    frameskip=frameskip, stack_frames=4, action_set=(1, 2, 3, 4),
                    score=(Term("reg", 6),), term=(), name=f"random-{seed}")


# --------------------------------------------------------------------------
# Super-CHIP workloads (the 128x64 variant): a hires template game and
# random-opcode programs over the CHIP-8 kinds plus the SCHIP forms.

PLAYER16_SPRITE = (0x07, 0xE0, 0x1F, 0xF8, 0x3F, 0xFC, 0x7F, 0xFE, 0x7F, 0xFE, 0xFF, 0xFF,
                   0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0x7F, 0xFE, 0x7F, 0xFE,
                   0x3F, 0xFC, 0x1F, 0xF8, 0x07, 0xE0, 0x00, 0x00)   # 16x16 disc


def schip_template_rom(p: TemplateParams) -> bytes:
    """Hires (128x64) variant of the template game: 16x16 player (DXY0) moved
    by 4 keys, an 8x4 object falling at a CXNN column, 8x3 decorative
    draw/erase pairs, the score drawn in 8x10 glyphs (FX33, FX65, FX30), and on
    every hit the score copied through the flag registers (FX75/FX85) and a
    left-then-right scroll (00FC, 00FB)."""
    rng = np.random.Generator(np.random.Philox(key=p.seed + 0x5C41))
    a = Asm()
    a.op(0x00FF)               # hires
    a.op(0x6800 | 56)          # V8 = player x
    a.op(0x6900 | 44)          # V9 = player y
    a.op(0x6600)               # V6 = score
    a.ref(0x2, "draw_score")
    a.op(0x6B00 | 8)           # VB = object y
    a.op(0xCA7F)               # VA = rnd & 127
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.ref(0xA, "player")
    a.op(0xD890)               # 16x16 player
    a.label("loop")
    a.ref(0xA, "player")
    a.op(0xD890)               # erase
    for key, upd in ((7, 0x78FE), (9, 0x7802), (5, 0x79FE), (8, 0x7902)):
        a.op(0x6500 | key)
        a.op(0xE5A1)
        a.op(upd)
    a.op(0x6E7F)
    a.op(0x88E2)               # V8 &= 127
    a.op(0x6E3F)
    a.op(0x89E2)               # V9 &= 63
    a.ref(0xA, "player")
    a.op(0xD890)
    scratch = (0x3, 0x7, 0xE)
    readable = (0x3, 0x7, 0xE, 0x6, 0x8, 0x9, 0xA, 0xB)
    for _ in range(p.alu_ops):
        kind = int(rng.integers(0, 13))
        x = int(scratch[rng.integers(0, 3)])
        y = int(readable[rng.integers(0, len(readable))])
        nn = int(rng.integers(0, 256))
        if kind == 0:
            a.op(0x6000 | x << 8 | nn)
        elif kind == 1:
            a.op(0x7000 | x << 8 | nn)
        elif kind in (2, 3):
            a.op((0x3000 if kind == 2 else 0x4000) | x << 8 | nn)
        else:
            sub = (0x0, 0x1, 0x2, 0x3, 0x4, 0x5, 0x6, 0x7, 0xE)[kind - 4]
            a.op(0x8000 | x << 8 | y << 4 | sub)
    if p.deco_pairs:
        a.ref(0xA, "deco")
        a.op(0x6300 | int(rng.integers(0, 120)))
        a.op(0x6700 | int(rng.integers(12, 50)))
        for _ in range(p.deco_pairs):
            a.op(0xD373)
            a.op(0xD373)
    a.ref(0xA, "object")
    a.op(0xDAB4)               # erase object
    a.op(0x7B00 | 2 * p.fall)  # fall
    a.op(0x6E3B)               # VE = 59
    a.op(0x8EB5)               # VE = 59 - VB, VF = (59 >= VB)
    a.op(0x3F00)
    a.ref(0x1, "no_respawn")
    a.op(0x6B00 | 8)
    a.op(0xCA7F)
    a.label("no_respawn")
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.op(0x3F00)
    a.ref(0x2, "hit")
    a.op(0x6400 | p.wait_frames)
    a.op(0xF415)
    a.label("wait")
    a.op(0xF407)
    a.op(0x3400)
    a.ref(0x1, "wait")
    a.ref(0x1, "loop")
    a.label("hit")
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.ref(0x2, "draw_score")   # erase
    a.op(0x7601)
    a.op(0xF675)               # flags[0..6] = V0..V6
    a.op(0x6600)
    a.op(0xF685)               # V0..V6 = flags[0..6] (score back)
    a.ref(0x2, "draw_score")
    a.op(0x00FC)               # scroll left 4 ...
    a.op(0x00FB)               # ... and back (edge columns lost)
    a.op(0x6B00 | 8)
    a.op(0xCA7F)
    a.ref(0xA, "object")
    a.op(0xDAB4)
    a.op(0x00EE)
    a.label("draw_score")
    a.ref(0xA, "scratch")
    a.op(0xF633)
    a.op(0xF265)
    a.op(0x6C00 | 98)
    a.op(0x6D00 | 1)
    for d in range(3):
        a.op(0xF030 | d << 8)  # I = 8x10 glyph of Vd
        a.op(0xDCDA)
        a.op(0x7C09)
    a.op(0x00EE)
    a.label("player")
    a.data(PLAYER16_SPRITE)
    a.label("object")
    a.data(OBJECT_SPRITE)
    a.label("deco")
    a.data(DECO_SPRITE)
    a.label("scratch")
    a.data((0, 0, 0, 0))
    rom = bytearray(a.assemble())
    if len(rom) < p.size:
        rom += rng.integers(0, 256, size=p.size - len(rom), dtype=np.uint8).tobytes()
    return bytes(rom)


def schip_template_game(p: TemplateParams, *, instr_per_frame: int = 20, frameskip: int = 4,
                        score_limit: int = 0, max_episode_steps: int = 0) -> GameSpec:
    """SCHIP template ROM + descriptor: reward = V6 increase, done at V6 >= limit."""
    term = (Clause(Term("reg", 6), ">=", score_limit),) if score_limit > 0 else ()
    return GameSpec(rom=schip_template_rom(p), instr_per_frame=instr_per_frame,
                    frameskip=frameskip, stack_frames=4, action_set=(7, 9, 5, 8),
                    score=(Term("reg", 6),), term=term,
                    max_episode_steps=max_episode_steps, startup_instrs=0, variant="schip",
                    name=f"schip-template-{p.seed}")


SCHIP_KINDS = ("00CN", "00FB", "00FC", "00FD", "00FE", "00FF", "DXY0", "FX30", "FX75", "FX85")


def random_schip_rom(seed: int, n_bytes: int = 3584, schip_weight: float = 0.15,
                     exit_weight: float = 0.002) -> bytes:
    """Random program over the 35 CHIP-8 kinds and the SCHIP forms: each
    opcode is a SCHIP form with probability ``schip_weight`` (00FD at
    ``exit_weight``, the rest uniform), otherwise a CHIP-8 opcode as in
    ``random_opcode_rom``."""
    base = bytearray(random_opcode_rom(seed, n_bytes))
    rng = np.random.Generator(np.random.Philox(key=seed + 0x5C42))
    n_ops = n_bytes // 2
    others = [k for k in SCHIP_KINDS if k != "00FD"]
    for i in range(n_ops):
        u = rng.random()
        if u < exit_weight:
            k = "00FD"
        elif u < schip_weight:
            k = others[int(rng.integers(0, len(others)))]
        else:
            continue
        x, y, n = int(rng.integers(0, 16)), int(rng.integers(0, 16)), int(rng.integers(0, 16))
        if k == "00CN":
            w = 0x00C0 | n
        elif k == "DXY0":
            w = 0xD000 | x << 8 | y << 4
        elif k[0] == "F":
            w = 0xF000 | x << 8 | int(k[2:], 16)
        else:
            w = int(k, 16)
        base[2 * i:2 * i + 2] = bytes((w >> 8, w & 0xFF))
    return bytes(base)


def random_schip_game(seed: int, *, instr_per_frame: int = 10, frameskip: int = 4) -> GameSpec:
    return GameSpec(rom=random_schip_rom(seed), instr_per_frame=instr_per_frame,
                    frameskip=frameskip, stack_frames=4, action_set=(1, 2, 3, 4),
                    score=(Term("reg", 6),), term=(), variant="schip", name=f"random-schip-{seed}")


# --------------------------------------------------------------------------
# Action streams: uniform over the action set, counter-based per step so that
# any window of steps can be regenerated independently.


# --------------------------------------------------------------------------
# Target Shooter, levels 1-3 (App. D): targets appear at random places, the
# player moves a crosshair onto them and shoots; each hit adds one to V2, and
# after ten targets V3 becomes 1. Level 1 targets stay until hit; level 2
# targets expire after a delay-timer timeout (a miss, which still counts
# towards the ten); level 3 targets also move, bouncing off the edges. Keys:
# 5 up, 8 down, 7 left, 9 right, 6 shoot. These programs are written here
# from that description and register mapping, not from the paper's listings.

CROSSHAIR_SPRITE = (0x20, 0x20, 0xF8, 0x20, 0x20)  # 5x5 plus, centre at (+2, +2)
TARGET_SPRITE = (0x70, 0xD8, 0xA8, 0xD8, 0x70)     # 5x5 ring with a centre dot
SHOOTER_TARGETS = 10
SHOOTER_KEYS = (5, 7, 8, 9, 6)                      # up, left, down, right, shoot


def shooter_rom(level: int, timeout_frames: int = 0) -> bytes:
    """Target Shooter ROM for level 1, 2 or 3 (see above)."""
    return _shooter(level, timeout_frames)[0]


def shooter_labels(level: int, timeout_frames: int = 0) -> dict:
    """Addresses of the Target Shooter labels (``loop``, ``shoot``, ``end`` ...)."""
    return _shooter(level, timeout_frames)[1]


def _shooter(level: int, timeout_frames: int) -> tuple:
    """Assemble one Target Shooter level.

    Registers: V0/V1 crosshair x/y, V2 score, V3 game-over flag, V4/V5 target
    x/y, V6 targets shown so far, V7/V8 target velocity (level 3), V9 key
    scratch, VA move phase (level 3), VB timeout, VC-VE scratch.
    timeout_frames: target lifetime in 60 Hz frames for levels 2 and 3
    (default 90 and 120).
    """
    assert level in (1, 2, 3)
    timeout = timeout_frames or (0, 0, 90, 120)[level]
    a = Asm()
    # ---- init
    a.op(0x6200)               # V2 = 0 (score)
    a.op(0x6300)               # V3 = 0
    a.op(0x6600)               # V6 = 0 (targets shown)
    a.op(0x6000 | 30)          # V0 = crosshair x
    a.op(0x6100 | 14)          # V1 = crosshair y
    a.op(0x6A00)               # VA = 0
    a.op(0x6B00 | timeout)     # VB = timeout
    a.ref(0x2, "draw_score")
    a.ref(0xA, "cross")
    a.op(0xD015)               # draw crosshair
    a.ref(0x2, "spawn")
    # ---- main loop
    a.label("loop")
    if level >= 2:             # expired target: a miss
        a.op(0xF907)           # V9 = DT
        a.op(0x3900)           # skip next if V9 == 0
        a.ref(0x1, "alive")
        a.ref(0x2, "miss")
        a.label("alive")
    if level == 3:             # move the target every second pass
        a.op(0x7A01)           # VA += 1
        a.op(0x6E01)
        a.op(0x8EA2)           # VE = VA & 1
        a.op(0x3E00)           # skip next if VE == 0
        a.ref(0x2, "move")
    a.ref(0xA, "cross")
    a.op(0xD015)               # erase crosshair
    for key, upd in ((5, 0x71FF), (8, 0x7101), (7, 0x70FF), (9, 0x7001)):
        a.op(0x6900 | key)     # V9 = key
        a.op(0xE9A1)           # skip next if key V9 is not held
        a.op(upd)              # move
    a.op(0x6E3F)
    a.op(0x80E2)               # V0 &= 63
    a.op(0x6E1F)
    a.op(0x81E2)               # V1 &= 31
    a.op(0xD015)               # redraw crosshair
    a.op(0x6906)               # V9 = shoot key
    a.op(0xE99E)               # skip next if held
    a.ref(0x1, "loop")
    a.ref(0x2, "shoot")
    a.ref(0x1, "loop")
    # ---- shoot: a hit when |V0 - V4| <= 2 and |V1 - V5| <= 2
    a.label("shoot")
    for p, t in ((0x0, 0x4), (0x1, 0x5)):
        a.op(0x8C00 | p << 4)  # VC = crosshair coordinate
        a.op(0x8C05 | t << 4)  # VC -= target coordinate
        a.op(0x7C02)           # VC += 2: 0..4 on a hit
        a.op(0x6D04)
        a.op(0x8DC5)           # VD = 4 - VC, VF = (4 >= VC)
        a.op(0x3F01)           # skip next if VF == 1
        a.op(0x00EE)           # out of range: return
    a.ref(0x2, "draw_score")   # erase old score
    a.op(0x7201)               # V2 += 1
    a.ref(0x2, "draw_score")   # draw new score
    a.ref(0x1, "next")
    # ---- miss: the target expired
    a.label("miss")
    # ---- next: erase the target, show the next one or end the game
    a.label("next")
    a.ref(0xA, "target")
    a.op(0xD455)               # erase target
    a.op(0x3600 | SHOOTER_TARGETS)  # skip next if V6 == 10
    a.ref(0x1, "spawn")        # (tail call: spawn returns to the caller)
    a.op(0x6301)               # V3 = 1: game over
    a.label("end")
    a.ref(0x1, "end")
    # ---- spawn: random place, reset the timer (and velocity), draw
    a.label("spawn")
    a.op(0xC437)               # V4 = rnd & 0x37
    a.op(0xC517)               # V5 = rnd & 0x17
    a.op(0x7402)               # V4 in 2..57
    a.op(0x7502)               # V5 in 2..25
    a.op(0x7601)               # V6 += 1
    if level >= 2:
        a.op(0xFB15)           # DT = VB
    if level == 3:
        for r in (0x7, 0x8):
            a.op(0xC002 | r << 8)  # Vr = rnd & 2
            a.op(0x70FF | r << 8)  # Vr -= 1: +1 or -1
    a.ref(0xA, "target")
    a.op(0xD455)               # draw target
    a.op(0x00EE)
    if level == 3:
        # ---- move: erase, step with bounces at x 1/58 and y 1/26, draw
        a.label("move")
        a.ref(0xA, "target")
        a.op(0xD455)
        for c, v, hi in ((0x4, 0x7, 58), (0x5, 0x8, 26)):
            a.op(0x8E00 | c << 4)      # VE = coordinate
            a.op(0x8E04 | v << 4)      # VE += velocity
            for edge in (1, hi):
                a.op(0x4E00 | edge)    # skip next if VE != edge
                a.ref(0x2, f"flip{v}")  # reverse the velocity
            a.op(0x8004 | c << 8 | v << 4)  # coordinate += velocity
        a.op(0xD455)
        a.op(0x00EE)
        for v in (0x7, 0x8):
            a.label(f"flip{v}")
            a.op(0x6D00)
            a.op(0x8D05 | v << 4)      # VD = 0 - velocity
            a.op(0x80D0 | v << 8)      # velocity = VD
            a.op(0x00EE)
    # ---- draw_score: hex digit of V2 at (59, 1)
    a.label("draw_score")
    a.op(0x6C00 | 59)
    a.op(0x6D01)
    a.op(0xF229)               # I = glyph(V2)
    a.op(0xDCD5)
    a.op(0x00EE)
    # ---- data
    a.label("cross")
    a.data(CROSSHAIR_SPRITE)
    a.label("target")
    a.data(TARGET_SPRITE)
    return a.assemble(), dict(a.labels)


def shooter_game(level: int, *, instr_per_frame: int = 10, frameskip: int = 4, timeout_frames: int = 0,
                 max_episode_steps: int = 0, sticky_prob: float = 0.0, max_noops: int = 0) -> GameSpec:
    """Target Shooter descriptor: reward = V2 increase (one per hit), done
    when V3 == 1, actions (up, left, down, right, shoot) = keys 5, 7, 8, 9, 6."""
    return GameSpec(rom=shooter_rom(level, timeout_frames), instr_per_frame=instr_per_frame,
                    frameskip=frameskip, stack_frames=4, action_set=SHOOTER_KEYS,
                    score=(Term("reg", 2),), term=(Clause(Term("reg", 3), "==", 1),),
                    max_episode_steps=max_episode_steps, sticky_prob=sticky_prob,
                    max_noops=max_noops, name=f"target-shooter-{level}")


def actions(seed: int, step_lo: int, step_hi: int, n_envs: int, n_actions: int = 4) -> np.ndarray:
    """uint8 [step_hi - step_lo, n_envs] drawn from Philox(seed, counter=step)."""
    out = np.empty((step_hi - step_lo, n_envs), dtype=np.uint8)
    for s in range(step_lo, step_hi):
        g = np.random.Generator(np.random.Philox(key=seed, counter=[s, 0, 0, 0]))
        out[s - step_lo] = g.integers(0, n_actions, size=n_envs, dtype=np.uint8)
    return out


def policy_params(seed: int, n_logits: int) -> dict:
    """Seeded float32 parameters for the §4.1 actor-critic network (random
    initialisation: normal with standard deviation sqrt(2 / fan_in) for the
    convolutions and hidden layers, sqrt(1 / fan_in) for the two output
    layers, biases uniform in [-0.1, 0.1]). Shapes: w1 [32,4,8,4]
    (out, frame, kx, ky), w2 [64,32,4,4], w3 [64,64,3,3], wa1 / wc1
    [256,1024] (input index = channel * 16 + x * 4 + y of the 64 x 4 x 4
    features), wa2 [n_logits,256], wc2 [256], matching biases; bc2 is a
    one-element array."""
    g = np.random.Generator(np.random.Philox(key=seed, counter=[0, 0, 0, 7]))

    def normal(shape, fan_in, gain=2.0):
        return (g.standard_normal(shape) * np.sqrt(gain / fan_in)).astype(np.float32)

    def bias(n):
        return g.uniform(-0.1, 0.1, size=n).astype(np.float32)

    return {
        "w1": normal((32, 4, 8, 4), 4 * 8 * 4), "b1": bias(32),
        "w2": normal((64, 32, 4, 4), 32 * 16), "b2": bias(64),
        "w3": normal((64, 64, 3, 3), 64 * 9), "b3": bias(64),
        "wa1": normal((256, 1024), 1024), "ba1": bias(256),
        "wa2": normal((n_logits, 256), 256, 1.0), "ba2": bias(n_logits),
        "wc1": normal((256, 1024), 1024), "bc1": bias(256),
        "wc2": normal((256,), 256, 1.0), "bc2": bias(1),
    }


# --------------------------------------------------------------------------
# The configurations the implementation is measured and checked on.


@dataclass
class Workload:
    name: str
    games: list
    game_of_env: np.ndarray | None  # uint16 [n_envs] or None (all game 0)
    n_envs: int
    n_steps: int
    seed: int
    quirks: int = 0
    action_seed: int = 1
    frames_per_launch: int = 4
    meta: dict = field(default_factory=dict)


def cfg_small() -> Workload:
    """64 instances of one ~600 B template ROM (seed 1), K = 10, frame skip 4,
    1,000 steps, no truncation."""
    g = template_game(TemplateParams(seed=1, size=600))
    return Workload("plain-small-64x1000", [g], None, 64, 1000, seed=1, action_seed=1)


def cfg_scale(n_envs: int = 16384, n_steps: int = 20000) -> Workload:
    """16,384 instances of a template ROM (seed 2), K = 10, frame skip 4,
    20,000 steps, done on score >= 20 or 5,000 steps (auto-reset)."""
    g = template_game(TemplateParams(seed=2, size=600), score_limit=20, max_episode_steps=5000)
    return Workload(f"plain-scale-{n_envs}x{n_steps}", [g], None, n_envs, n_steps, seed=2,
                    action_seed=2)


def cfg_wrappers(n_envs: int = 16384, n_steps: int = 20000) -> Workload:
    """The 16,384-instance template workload behind the §3.2 wrappers: sticky
    actions with p = 0.25 and no-op resets of 0-30 steps (the values commonly
    used for Atari agents)."""
    w = cfg_scale(n_envs, n_steps)
    g = replace(w.games[0], sticky_prob=0.25, max_noops=30)
    return Workload(f"wrappers-scale-{n_envs}x{n_steps}", [g], None, n_envs, n_steps, seed=w.seed,
                    action_seed=w.action_seed)


def cfg_schip(n_envs: int = 16384, n_steps: int = 4000) -> Workload:
    """16,384 instances of the hires SCHIP template ROM (seed 3), K = 20, frame
    skip 4, observations uint8 [4, 64, 128], done on score >= 20 or 2,000 steps."""
    g = schip_template_game(TemplateParams(seed=3, size=700, deco_pairs=1), score_limit=20,
                            max_episode_steps=2000)
    return Workload(f"schip-scale-{n_envs}x{n_steps}", [g], None, n_envs, n_steps, seed=3,
                    action_seed=3)


def cfg_shooter(n_envs: int = 16384, n_steps: int = 20000) -> Workload:
    """16,384 instances of the three Target Shooter levels (instance i plays
    level 1 + i mod 3), K = 10, frame skip 4, uniform random actions over the
    five actions, done after ten targets or 5,000 steps (auto-reset)."""
    games = [shooter_game(level, max_episode_steps=5000) for level in (1, 2, 3)]
    goe = (np.arange(n_envs) % 3).astype(np.uint16)
    return Workload(f"target-shooter-{n_envs}x{n_steps}", games, goe, n_envs, n_steps, seed=5,
                    action_seed=5)


BATCH_K = (5, 8, 10, 15, 20)


def cfg_batch(n_envs: int = 65536, n_steps: int = 4000) -> Workload:
    """65,536 instances over 16 template ROMs (seeds 100-115), 200-3,000 B,
    DXYN share ~5-40 %, K per ROM from {5, 8, 10, 15, 20}, termination
    threshold per ROM from 5..40, truncation 5,000; 16 frames per launch."""
    rng = np.random.Generator(np.random.Philox(key=777))
    games = []
    for i in range(16):
        seed = 100 + i
        size = int(200 + (3000 - 200) * i / 15)
        # DXYN share rises with i: more draw/erase pairs, less ALU filler
        deco = i
        alu = (15 - i) + int(rng.integers(0, 9))
        wait = int(rng.integers(0, 3))
        k = int(BATCH_K[int(rng.integers(0, len(BATCH_K)))])
        limit = int(rng.integers(5, 41))
        p = TemplateParams(seed=seed, size=size, alu_ops=alu, deco_pairs=deco,
                           wait_frames=wait, fall=1 + int(rng.integers(0, 2)))
        rom = template_rom(p)
        if len(rom) > size:        # code longer than the target: keep the code
            p = replace(p, size=len(rom))
        games.append(template_game(p, instr_per_frame=k, score_limit=limit,
                                   max_episode_steps=5000))
    # uneven instance counts per ROM, interleaved instance order
    w = rng.uniform(0.25, 1.75, size=16)
    counts = np.floor(w / w.sum() * n_envs).astype(np.int64)
    counts[0] += n_envs - counts.sum()
    game_of_env = np.repeat(np.arange(16, dtype=np.uint16), counts)
    rng.shuffle(game_of_env)
    return Workload(f"batch-{n_envs}x{n_steps}-16roms", games, game_of_env, n_envs, n_steps,
                    seed=3, action_seed=3, frames_per_launch=16)


def cfg_divergence(n_envs: int = 262144, n_steps: int = 2000, n_roms: int = 64) -> Workload:
    """262,144 instances of random-opcode ROMs (3,584 B, CXNN at 10 %),
    K = 10, frame skip 4, 2,000 steps; instance i runs ROM i % 64."""
    games = [random_game(1000 + r) for r in range(n_roms)]
    game_of_env = (np.arange(n_envs) % n_roms).astype(np.uint16)
    return Workload(f"divergence-{n_envs}x{n_steps}", games, game_of_env, n_envs, n_steps,
                    seed=4, action_seed=4)
