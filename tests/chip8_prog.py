"""Helpers for hand-assembled test programs (raw opcode words)."""
from paper_2510_01764_gb300.workloads import Clause, GameSpec, Term


def rom(words, data=b"") -> bytes:
    return b"".join(bytes(((w >> 8) & 0xFF, w & 0xFF)) for w in words) + bytes(data)


def prog(words, data=b"", **kw) -> GameSpec:
    kw.setdefault("action_set", (7, 9, 5, 8))
    return GameSpec(rom=rom(words, data), **kw)


# Register maps of the paper's games (§3.3, App. C game list, App. F wrapper).
# Expressions are restated as descriptor terms/clauses; the tests evaluate the
# paper's own Python expressions next to them.
PAPER_GAMES = {
    "tetris": ((Term("reg", 10),), (Clause(Term("reg", 1), "==", 2),)),
    "blinky": ((Term("reg", 6),), (Clause(Term("reg", 3), "==", 255),)),
    "worm": ((Term("reg", 5),), (Clause(Term("reg", 7), "==", 255),)),
    "brix": ((Term("reg", 5),), (Clause(Term("reg", 14), "==", 4),)),
    "pong": ((Term("reg", 14, "dec_tens_minus_ones"),),
             (Clause(Term("reg", 14, "dec_tens"), "==", 9),
              Clause(Term("reg", 14, "dec_ones"), "==", 9))),
    "squash": ((Term("reg", 11),), (Clause(Term("reg", 11), "==", 0),)),
    "vertical_brix": ((Term("reg", 8),), (Clause(Term("reg", 7), "==", 0),)),
    "wipe_off": ((Term("reg", 6),), (Clause(Term("reg", 7), "==", 0),)),
    "filter": ((Term("reg", 14),), (Clause(Term("reg", 13), "==", 0),)),
    "missile": ((Term("reg", 7),), (Clause(Term("reg", 6), "==", 0),)),
    "rocket": ((Term("reg", 1),), (Clause(Term("reg", 2), "==", 9),)),
    "submarine": ((Term("reg", 7),), (Clause(Term("reg", 8), "==", 0),)),
    "tank": ((Term("reg", 14),), (Clause(Term("reg", 6), "==", 0),)),
    "ufo": ((Term("reg", 7),), (Clause(Term("reg", 8), "==", 0),)),
    "cavern": ((Term("reg", 0),), (Clause(Term("reg", 14), "==", 0),)),
    "flight_runner": ((Term("reg", 7),), (Clause(Term("reg", 5), "==", 255),
                                          Clause(Term("reg", 7), "==", 255))),
    "space_flight": ((Term("reg", 0),), (Clause(Term("reg", 9), "==", 0),
                                         Clause(Term("reg", 12), ">=", 0x3E))),
    "spacejam": ((Term("reg", 9),), (Clause(Term("reg", 10), "==", 0),)),
    "airplane": ((Term("reg", 11, "neg"), Term("reg", 12, "neg")),
                 (Clause(Term("reg", 11), "==", 0), Clause(Term("reg", 12), "==", 6))),
    "deep": ((Term("reg", 9),), (Clause(Term("reg", 11), "!=", 1),)),
    "shooting_stars": ((Term("reg", 0, "zero_if_gt", 128),), ()),
    "target_shooter": ((Term("reg", 2),), (Clause(Term("reg", 3), "==", 1),)),
}

# The paper's expressions, as printed (§3.3 and App. C / App. F), over V.
PAPER_EXPR = {
    "tetris": (lambda V: V[10], lambda V: V[1] == 2),
    "blinky": (lambda V: V[6], lambda V: V[3] == 255),
    "worm": (lambda V: V[5], lambda V: V[7] == 255),
    "brix": (lambda V: V[5], lambda V: V[14] == 4),
    "pong": (lambda V: (V[14] // 10) - (V[14] % 10),
             lambda V: (V[14] // 10) == 9 or (V[14] % 10) == 9),
    "squash": (lambda V: V[11], lambda V: V[11] == 0),
    "vertical_brix": (lambda V: V[8], lambda V: V[7] == 0),
    "wipe_off": (lambda V: V[6], lambda V: V[7] == 0),
    "filter": (lambda V: V[14], lambda V: V[13] == 0),
    "missile": (lambda V: V[7], lambda V: V[6] == 0),
    "rocket": (lambda V: V[1], lambda V: V[2] == 9),
    "submarine": (lambda V: V[7], lambda V: V[8] == 0),
    "tank": (lambda V: V[14], lambda V: V[6] == 0),
    "ufo": (lambda V: V[7], lambda V: V[8] == 0),
    "cavern": (lambda V: V[0], lambda V: V[14] == 0),
    "flight_runner": (lambda V: V[7], lambda V: V[5] == 255 or V[7] == 255),
    "space_flight": (lambda V: V[0], lambda V: V[9] == 0 or V[12] >= 0x3E),
    "spacejam": (lambda V: V[9], lambda V: V[10] == 0),
    "airplane": (lambda V: -V[11] - V[12], lambda V: V[11] == 0 or V[12] == 6),
    "deep": (lambda V: V[9], lambda V: V[11] != 1),
    "shooting_stars": (lambda V: 0 if V[0] > 128 else V[0], lambda V: False),
    "target_shooter": (lambda V: V[2], lambda V: V[3] == 1),
}
