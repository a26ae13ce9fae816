"""ctypes binding of the plain-C CHIP-8 environment oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package. It
shares no code with the CUDA path; games arrive as
``paper_2510_01764_gb300.workloads.GameSpec``-shaped objects (duck-typed, read
attribute by attribute) and are marshalled into the oracle's own structs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "octax_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboctax_oracle.so")
_lock = threading.Lock()
_lib = None

QUIRKS = {"shift_uses_vy": 0x01, "loadstore_inc_i": 0x02, "logic_resets_vf": 0x04,
          "jump_vx": 0x08, "wrap_sprites": 0x10, "fx1e_vf": 0x20}
ST_BAD_OP, ST_STACK_FAULT, ST_BAD_ACTION, ST_EXIT = 1, 2, 4, 8
VARIANTS = {"chip8": 0, "schip": 1}


def frame_shape(variant: str) -> tuple:
    """(rows, columns) of one observation frame."""
    return (64, 128) if variant == "schip" else (32, 64)

_XFORM = {"raw": 0, "neg": 1, "dec_tens": 2, "dec_ones": 3, "dec_tens_minus_ones": 4,
          "nib_hi_minus_lo": 5, "zero_if_gt": 6}
_CMP = {"==": 0, "!=": 1, ">=": 2, ">": 3, "<=": 4, "<": 5}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, plain C, pthreads)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "octax_oracle.h")]
    if not force and os.path.exists(_LIB) and all(
            os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in srcs):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lpthread"])
    os.replace(tmp, _LIB)
    return _LIB


class Term(C.Structure):
    _fields_ = [("src", C.c_int32), ("idx", C.c_int32), ("xform", C.c_int32), ("arg", C.c_int32)]


class Clause(C.Structure):
    _fields_ = [("lhs", Term), ("cmp", C.c_int32), ("rhs", C.c_int32)]


class Game(C.Structure):
    _fields_ = [("rom", C.POINTER(C.c_uint8)), ("rom_len", C.c_uint32),
                ("instr_per_frame", C.c_uint32), ("frameskip", C.c_uint32),
                ("stack_frames", C.c_uint32), ("n_actions", C.c_uint32),
                ("action_set", C.c_uint8 * 16), ("n_score_terms", C.c_uint32),
                ("score", Term * 4), ("n_term_clauses", C.c_uint32), ("term", Clause * 4),
                ("max_episode_steps", C.c_uint32), ("startup_instrs", C.c_uint32),
                ("sticky_threshold", C.c_uint32), ("max_noops", C.c_uint32),
                ("variant", C.c_uint32)]


class Inst(C.Structure):
    _fields_ = [("V", C.c_uint8 * 16), ("I", C.c_uint16), ("PC", C.c_uint16), ("SP", C.c_uint8),
                ("DT", C.c_uint8), ("ST", C.c_uint8), ("status", C.c_uint8),
                ("stack", C.c_uint16 * 16), ("pix", (C.c_uint8 * 128) * 64),
                ("ram", C.c_uint8 * 4096), ("episode_steps", C.c_uint32),
                ("env_steps", C.c_uint32), ("key", C.c_uint32 * 2), ("uid", C.c_uint32),
                ("phase", C.c_uint32), ("draws", C.c_uint32), ("game", C.c_int32),
                ("last_action", C.c_uint8), ("variant", C.c_uint8), ("hires", C.c_uint8),
                ("rpl", C.c_uint8 * 16)]


RECORD_DTYPE = np.dtype([("V", np.uint8, 16), ("I", "<u2"), ("PC", "<u2"), ("SP", np.uint8),
                         ("DT", np.uint8), ("ST", np.uint8), ("status", np.uint8),
                         ("stack", "<u2", 16), ("display", "<u8", (64, 2)), ("ram", np.uint8, 4096),
                         ("episode_steps", "<u4"), ("env_steps", "<u4"), ("last_action", np.uint8),
                         ("hires", np.uint8), ("pad", np.uint8, 6), ("rpl", np.uint8, 16)])
assert RECORD_DTYPE.itemsize == 5208


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_fnv1a64.argtypes = [P, C.c_size_t]
            L.orc_fnv1a64.restype = C.c_uint64
            L.orc_inst_reset.argtypes = [C.POINTER(Inst), C.POINTER(Game), C.c_uint32]
            L.orc_exec_one.argtypes = [C.POINTER(Inst), C.c_uint32, C.c_int]
            L.orc_tick_timers.argtypes = [C.POINTER(Inst)]
            L.orc_score.argtypes = [C.POINTER(Inst), C.POINTER(Game)]
            L.orc_score.restype = C.c_int32
            L.orc_terminated.argtypes = [C.POINTER(Inst), C.POINTER(Game)]
            L.orc_inst_step.argtypes = [C.POINTER(Inst), C.POINTER(Game), C.c_uint32, C.c_uint32,
                                        P, C.POINTER(C.c_float), C.POINTER(C.c_uint8)]
            L.orc_inst_record.argtypes = [C.POINTER(Inst), P]
            L.orc_inst_hash.argtypes = [C.POINTER(Inst)]
            L.orc_inst_hash.restype = C.c_uint64
            L.orc_env_create.argtypes = [C.POINTER(Game), C.c_int, P, P, C.c_int64, C.c_uint32,
                                         C.c_uint64]
            L.orc_env_create.restype = P
            L.orc_env_reset.argtypes = [P, P, P]
            L.orc_env_step.argtypes = [P, P, P, P, P, C.c_int]
            L.orc_env_hash.argtypes = [P, P]
            L.orc_env_records.argtypes = [P, P]
            L.orc_env_inst.argtypes = [P, C.c_int64]
            L.orc_env_inst.restype = C.POINTER(Inst)
            L.orc_env_destroy.argtypes = [P]
            L.orc_env_rollout.argtypes = [P, C.c_int, P, P, P, P, P, C.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _term(t) -> Term:
    return Term(0 if t.src == "reg" else 1, int(t.idx), _XFORM[t.xform], int(t.arg))


def make_game(spec) -> tuple[Game, object]:
    """Marshal a GameSpec-like object; returns (struct, keep-alive buffer)."""
    rom = np.frombuffer(bytes(spec.rom), dtype=np.uint8).copy()
    g = Game()
    g.rom = rom.ctypes.data_as(C.POINTER(C.c_uint8))
    g.rom_len = len(rom)
    g.instr_per_frame = spec.instr_per_frame
    g.frameskip = spec.frameskip
    g.stack_frames = spec.stack_frames
    g.n_actions = len(spec.action_set)
    for i, k in enumerate(spec.action_set):
        g.action_set[i] = k
    g.n_score_terms = len(spec.score)
    for i, t in enumerate(spec.score):
        g.score[i] = _term(t)
    g.n_term_clauses = len(spec.term)
    for i, c in enumerate(spec.term):
        g.term[i] = Clause(_term(c.lhs), _CMP[c.cmp], int(c.rhs))
    g.max_episode_steps = spec.max_episode_steps
    g.startup_instrs = spec.startup_instrs
    g.sticky_threshold = sticky_threshold(getattr(spec, "sticky_prob", 0.0))
    g.max_noops = getattr(spec, "max_noops", 0)
    g.variant = VARIANTS[getattr(spec, "variant", "chip8")]
    return g, rom


def sticky_threshold(p: float) -> int:
    """Probability -> 32-bit threshold (repeat when a uniform draw is below it)."""
    return min(int(round(float(p) * 2 ** 32)), 2 ** 32 - 1) if p > 0 else 0


def philox4x32_10(ctr, key) -> tuple:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return tuple(int(v) for v in out)


def fnv1a64(data: bytes) -> int:
    buf = np.frombuffer(data, dtype=np.uint8).copy()
    return int(lib().orc_fnv1a64(_ptr(buf), len(buf)))


class Machine:
    """One oracle instance driven instruction by instruction (unit tests)."""

    def __init__(self, spec, quirks: int = 0, seed: int = 0, uid: int = 0):
        self._g, self._rom = make_game(spec)
        self._variant = getattr(spec, "variant", "chip8")
        self.quirks = quirks
        self.m = Inst()
        self.m.key[0] = seed & 0xFFFFFFFF
        self.m.key[1] = seed >> 32
        self.m.uid = uid
        rc = lib().orc_inst_reset(C.byref(self.m), C.byref(self._g), quirks)
        assert rc == 0

    def exec(self, n: int = 1, key: int = -1) -> None:
        for _ in range(n):
            lib().orc_exec_one(C.byref(self.m), self.quirks, key)

    def tick(self) -> None:
        lib().orc_tick_timers(C.byref(self.m))

    def step(self, action: int, obs: bool = True):
        o = np.zeros((self._g.stack_frames,) + frame_shape(self._variant), dtype=np.uint8) if obs else None
        r = C.c_float()
        d = C.c_uint8()
        lib().orc_inst_step(C.byref(self.m), C.byref(self._g), self.quirks, action, _ptr(o),
                            C.byref(r), C.byref(d))
        return o, r.value, d.value

    def score(self) -> int:
        return lib().orc_score(C.byref(self.m), C.byref(self._g))

    def terminated(self) -> bool:
        return bool(lib().orc_terminated(C.byref(self.m), C.byref(self._g)))

    @property
    def V(self) -> list:
        return list(self.m.V)

    def set_V(self, i: int, v: int) -> None:
        self.m.V[i] = v

    @property
    def pixels(self) -> np.ndarray:
        """The screen: 32x64 (CHIP-8) or the 64x128 buffer (SCHIP)."""
        h, w = frame_shape(self._variant)
        return np.ctypeslib.as_array(self.m.pix)[:h, :w].copy()

    @property
    def ram(self) -> np.ndarray:
        return np.ctypeslib.as_array(self.m.ram).copy()

    def record(self) -> np.ndarray:
        out = np.zeros(1, dtype=RECORD_DTYPE)
        lib().orc_inst_record(C.byref(self.m), _ptr(out))
        return out[0]

    def hash(self) -> int:
        return int(lib().orc_inst_hash(C.byref(self.m)))


class OracleEnv:
    """A batch of independent oracle instances (the loop over environments)."""

    def __init__(self, games, n_envs: int, *, game_of_env=None, uid_of_env=None,
                 quirks: int = 0, seed: int = 0):
        self._keep = [make_game(g) for g in games]
        arr = (Game * len(games))(*[k[0] for k in self._keep])
        self._games_arr = arr
        self.n = int(n_envs)
        self.stack_frames = games[0].stack_frames
        self.frame = frame_shape(getattr(games[0], "variant", "chip8"))
        self._goe = None if game_of_env is None else np.ascontiguousarray(game_of_env, dtype=np.uint16)
        self._uoe = None if uid_of_env is None else np.ascontiguousarray(uid_of_env, dtype=np.uint32)
        self.h = lib().orc_env_create(arr, len(games), _ptr(self._goe), _ptr(self._uoe), self.n,
                                      quirks, seed)
        if not self.h:
            raise ValueError("oracle rejected the environment description")

    def close(self) -> None:
        if self.h:
            lib().orc_env_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def reset(self, mask=None) -> np.ndarray:
        obs = np.zeros((self.n, self.stack_frames) + self.frame, dtype=np.uint8)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        lib().orc_env_reset(self.h, _ptr(m), _ptr(obs))
        return obs

    def step(self, actions, *, obs: bool = True, threads: int = 1):
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        assert a.shape == (self.n,)
        o = np.zeros((self.n, self.stack_frames) + self.frame, dtype=np.uint8) if obs else None
        r = np.zeros(self.n, dtype=np.float32)
        d = np.zeros(self.n, dtype=np.uint8)
        lib().orc_env_step(self.h, _ptr(a), _ptr(o), _ptr(r), _ptr(d), threads)
        return o, r, d

    def rollout(self, actions, *, obs: bool = False, hashes: bool = False, threads: int = 1):
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        steps = a.shape[0]
        assert a.shape[1] == self.n
        o = np.zeros((steps, self.n, self.stack_frames) + self.frame, dtype=np.uint8) if obs else None
        r = np.zeros((steps, self.n), dtype=np.float32)
        d = np.zeros((steps, self.n), dtype=np.uint8)
        h = np.zeros((steps, self.n), dtype=np.uint64) if hashes else None
        lib().orc_env_rollout(self.h, steps, _ptr(a), _ptr(o), _ptr(r), _ptr(d), _ptr(h), threads)
        return o, r, d, h

    def hashes(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.uint64)
        lib().orc_env_hash(self.h, _ptr(out))
        return out

    def records(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=RECORD_DTYPE)
        lib().orc_env_records(self.h, _ptr(out))
        return out

    def inst(self, i: int) -> Inst:
        return lib().orc_env_inst(self.h, i).contents
