"""Python binding of liboctax (include/octax.h): argument marshalling only.

Every step of the environment runs in the hand-written CUDA kernels of the
in-tree ``_build/liboctax.so``; this module converts game descriptions into
the C structs, allocates output tensors with PyTorch and passes raw pointers
and the CUDA stream. There is no CPU fallback: if the library is missing the
import of ``Env`` fails with instructions to build it.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liboctax.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTFOUND = 0, -1, -2, -3, -4, -5
QUIRK_SHIFT_USES_VY, QUIRK_LOADSTORE_INC_I, QUIRK_LOGIC_RESETS_VF = 0x01, 0x02, 0x04
QUIRK_JUMP_VX, QUIRK_WRAP_SPRITES, QUIRK_FX1E_VF = 0x08, 0x10, 0x20
STATUS_BAD_OP, STATUS_STACK_FAULT, STATUS_BAD_ACTION = 0x01, 0x02, 0x04

_XFORM = {"raw": 0, "neg": 1, "dec_tens": 2, "dec_ones": 3, "dec_tens_minus_ones": 4,
          "nib_hi_minus_lo": 5, "zero_if_gt": 6}
_CMP = {"==": 0, "!=": 1, ">=": 2, ">": 3, "<=": 4, "<": 5}


class OctaxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liboctax error {code}: {msg}")
        self.code = code


class CTerm(C.Structure):
    _fields_ = [("src", C.c_uint8), ("xform", C.c_uint8), ("idx", C.c_uint16), ("arg", C.c_int32)]


class CClause(C.Structure):
    _fields_ = [("lhs", CTerm), ("cmp", C.c_uint8), ("pad", C.c_uint8 * 3), ("rhs", C.c_int32)]


class CGame(C.Structure):
    _fields_ = [("rom", C.POINTER(C.c_uint8)), ("rom_len", C.c_uint32),
                ("instr_per_frame", C.c_uint8), ("frameskip", C.c_uint8),
                ("stack_frames", C.c_uint8), ("n_actions", C.c_uint8),
                ("action_set", C.c_uint8 * 16), ("n_score_terms", C.c_uint8),
                ("n_term_clauses", C.c_uint8), ("variant", C.c_uint8), ("pad", C.c_uint8),
                ("score", CTerm * 4),
                ("term", CClause * 4), ("max_episode_steps", C.c_uint32),
                ("startup_instrs", C.c_uint32), ("sticky_threshold", C.c_uint32),
                ("max_noops", C.c_uint32)]


class CLaunch(C.Structure):
    _fields_ = [("block", C.c_int32), ("inst_per_warp", C.c_int32),
                ("steps_per_launch", C.c_int32), ("persistent", C.c_int32),
                ("use_graph", C.c_int32), ("writer_warps", C.c_int32), ("balance", C.c_int32)]


RECORD_DTYPE = np.dtype([("V", np.uint8, 16), ("I", "<u2"), ("PC", "<u2"), ("SP", np.uint8),
                         ("DT", np.uint8), ("ST", np.uint8), ("status", np.uint8),
                         ("stack", "<u2", 16), ("display", "<u8", (64, 2)), ("ram", np.uint8, 4096),
                         ("episode_steps", "<u4"), ("env_steps", "<u4"),
                         ("last_action", np.uint8), ("hires", np.uint8), ("pad", np.uint8, 6),
                         ("rpl", np.uint8, 16)])
assert RECORD_DTYPE.itemsize == 5208
VARIANT_CHIP8, VARIANT_SCHIP = 0, 1
STATUS_EXIT = 0x08


def frame_shape(variant) -> tuple:
    """(rows, columns) of one observation frame of a variant ("chip8"/"schip" or 0/1)."""
    return (64, 128) if variant in ("schip", VARIANT_SCHIP) else (32, 64)

class CPolicyParams(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("w1", "b1", "w2", "b2", "w3", "b3", "wa1", "ba1", "wa2", "ba2",
                                          "wc1", "bc1", "wc2", "bc2")] + [("n_logits", C.c_int32)]


class CServerConfig(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_int64), ("block", C.c_int32),
                ("inst_per_warp", C.c_int32), ("max_inflight_ticks", C.c_int32),
                ("reserved", C.c_int32)]


class CRequest(C.Structure):
    _fields_ = [("game", C.c_uint16), ("pad", C.c_uint16), ("n_envs", C.c_uint32),
                ("n_steps", C.c_uint32), ("pad2", C.c_uint32), ("seed", C.c_uint64),
                ("actions_host", C.c_void_p), ("obs_dev", C.c_void_p),
                ("reward_dev", C.c_void_p), ("done_dev", C.c_void_p)]


class CRequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("pad", C.c_int32), ("submit_ns", C.c_int64),
                ("admit_ns", C.c_int64), ("done_ns", C.c_int64)]


class CServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "completed", "env_steps", "ticks",
                                         "peak_active_envs", "peak_active_requests",
                                         "slots_capacity", "slots_in_use", "queued")]


EXPORTS = ("octax_create", "octax_reset", "octax_step", "octax_step_n", "octax_step_host",
           "octax_state_hash", "octax_get_state", "octax_set_state", "octax_sync",
           "octax_get_launch", "octax_set_launch", "octax_autotune", "octax_num_envs",
           "octax_stack_frames", "octax_variant", "octax_step_n_packed", "octax_step_host_packed", "octax_debug_stall_writers", "octax_device_bytes", "octax_destroy", "octax_last_error",
           "octax_server_create", "octax_server_submit", "octax_server_wait",
           "octax_server_query", "octax_server_release", "octax_server_get_stats",
           "octax_server_destroy", "octax_server_submit_batch", "octax_server_wait_batch", "octax_rollout_static", "octax_policy_create", "octax_policy_forward",
           "octax_policy_forward_u8", "octax_rollout_policy", "octax_policy_sync", "octax_policy_debug_stall",
           "octax_policy_destroy")

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load liboctax.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} not found: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(path)
        P, I64, I32 = C.c_void_p, C.c_int64, C.c_int
        sig = {
            "octax_create": (I32, [C.POINTER(CGame), I32, P, P, I64, C.c_uint32, C.c_uint64, P,
                                   C.POINTER(P)]),
            "octax_reset": (I32, [P, P, P]),
            "octax_step": (I32, [P, P, P, P, P]),
            "octax_step_n": (I32, [P, I32, P, P, P, P]),
            "octax_step_host": (I32, [P, P, P, P, P]),
            "octax_step_n_packed": (I32, [P, I32, P, P, P, P]),
            "octax_step_host_packed": (I32, [P, P, P, P, P]),
            "octax_debug_stall_writers": (I32, [P, I32]),
            "octax_state_hash": (I32, [P, P]),
            "octax_get_state": (I32, [P, I64, I64, P]),
            "octax_set_state": (I32, [P, I64, I64, P]),
            "octax_sync": (I32, [P, I32]),
            "octax_get_launch": (I32, [P, C.POINTER(CLaunch)]),
            "octax_set_launch": (I32, [P, C.POINTER(CLaunch)]),
            "octax_autotune": (I32, [P, I32, P, C.POINTER(C.c_float)]),
            "octax_num_envs": (I64, [P]),
            "octax_stack_frames": (I32, [P]),
            "octax_variant": (I32, [P]),
            "octax_device_bytes": (C.c_size_t, [P]),
            "octax_destroy": (None, [P]),
            "octax_last_error": (C.c_char_p, []),
            "octax_server_create": (I32, [C.POINTER(CGame), I32, C.c_uint32,
                                          C.POINTER(CServerConfig), C.POINTER(P)]),
            "octax_server_submit": (I32, [P, C.POINTER(CRequest), C.POINTER(C.c_uint64)]),
            "octax_server_submit_batch": (I32, [P, C.POINTER(CRequest), I32, C.POINTER(C.c_uint64)]),
            "octax_server_wait_batch": (I32, [P, C.POINTER(C.c_uint64), I32, I32, C.POINTER(CRequestInfo), I32]),
            "octax_server_wait": (I32, [P, C.c_uint64, I32, C.POINTER(CRequestInfo)]),
            "octax_server_query": (I32, [P, C.c_uint64, C.POINTER(CRequestInfo)]),
            "octax_server_release": (I32, [P, C.c_uint64]),
            "octax_server_get_stats": (I32, [P, C.POINTER(CServerStats)]),
            "octax_server_destroy": (None, [P]),
            "octax_rollout_static": (I32, [C.POINTER(CGame), I64, C.c_uint32, C.c_uint64, I32,
                                           P, P, P, P, P]),
            "octax_policy_create": (I32, [C.POINTER(CPolicyParams), I64, I32, P, C.POINTER(P)]),
            "octax_policy_forward": (I32, [P, I64, P, C.c_uint64, C.c_uint32, P, P, P]),
            "octax_policy_forward_u8": (I32, [P, I64, P, C.c_uint64, C.c_uint32, P, P, P]),
            "octax_rollout_policy": (I32, [P, P, I32, C.c_uint64, C.c_uint32, P, P, P, P, P, P]),
            "octax_policy_sync": (I32, [P]),
            "octax_policy_debug_stall": (I32, [P, I32]),
            "octax_policy_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(rc: int) -> None:
    if rc != OK:
        raise OctaxError(rc, load_library().octax_last_error().decode())


def _term(t) -> CTerm:
    return CTerm(0 if t.src == "reg" else 1, _XFORM[t.xform], int(t.idx) & 0xFFFF, int(t.arg))


def make_game(spec) -> tuple[CGame, object]:
    """Marshal a GameSpec-like object into an octax_game (+ keep-alive buffer)."""
    rom = np.frombuffer(bytes(spec.rom), dtype=np.uint8).copy()
    g = CGame()
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
        g.term[i] = CClause(_term(c.lhs), _CMP[c.cmp], (C.c_uint8 * 3)(), int(c.rhs))
    g.max_episode_steps = spec.max_episode_steps
    g.startup_instrs = spec.startup_instrs
    g.sticky_threshold = sticky_threshold(getattr(spec, "sticky_prob", 0.0))
    g.max_noops = getattr(spec, "max_noops", 0)
    g.variant = VARIANT_SCHIP if getattr(spec, "variant", "chip8") == "schip" else VARIANT_CHIP8
    return g, rom


def sticky_threshold(p: float) -> int:
    """Sticky-action probability -> the descriptor's 32-bit threshold."""
    return min(int(round(float(p) * 2 ** 32)), 2 ** 32 - 1) if p > 0 else 0


def _ptr(t) -> C.c_void_p | None:
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


class Env:
    """n_envs CHIP-8 (or Super-CHIP) environments stepped by the CUDA kernels on one GPU."""

    def __init__(self, games, n_envs: int, *, game_of_env=None, uid_of_env=None,
                 quirks: int = 0, seed: int = 0, device=None, stream=None):
        import torch

        self._torch = torch
        L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("liboctax needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.games = list(games)
        self.n = int(n_envs)
        self.S = int(self.games[0].stack_frames)
        self.frame = frame_shape(getattr(self.games[0], "variant", "chip8"))
        keep = [make_game(g) for g in self.games]
        arr = (CGame * len(keep))(*[k[0] for k in keep])
        goe = None if game_of_env is None else np.ascontiguousarray(game_of_env, dtype=np.uint16)
        uoe = None if uid_of_env is None else np.ascontiguousarray(uid_of_env, dtype=np.uint32)
        if goe is not None and goe.shape != (self.n,):
            raise ValueError("game_of_env must have shape (n_envs,)")
        if uoe is not None and uoe.shape != (self.n,):
            raise ValueError("uid_of_env must have shape (n_envs,)")
        h = C.c_void_p()
        check(L.octax_create(arr, len(keep), None if goe is None else C.c_void_p(goe.ctypes.data),
                             None if uoe is None else C.c_void_p(uoe.ctypes.data), self.n, quirks,
                             seed & 0xFFFFFFFFFFFFFFFF, C.c_void_p(self.stream.cuda_stream),
                             C.byref(h)))
        self._h = h
        self._keep = keep

    # ------------------------------------------------------------------ helpers
    def _u8(self, *shape):
        return self._torch.empty(shape, dtype=self._torch.uint8, device=self.device)

    def _check_dev(self, t, dtype, shape, name):
        if t.device != self.device or t.dtype != dtype or tuple(t.shape) != tuple(shape) \
                or not t.is_contiguous():
            raise ValueError(f"{name}: need contiguous {dtype} {tuple(shape)} on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")

    @property
    def obs_shape(self):
        return (self.n, self.S) + self.frame

    # ------------------------------------------------------------------ API
    def reset(self, mask=None, out=None):
        torch = self._torch
        obs = out if out is not None else self._u8(*self.obs_shape)
        self._check_dev(obs, torch.uint8, self.obs_shape, "obs")
        if mask is not None:
            mask = mask.to(device=self.device, dtype=torch.uint8).contiguous()
            self._check_dev(mask, torch.uint8, (self.n,), "mask")
        check(load_library().octax_reset(self._h, _ptr(mask), _ptr(obs)))
        return obs

    def step(self, actions, out=None):
        torch = self._torch
        self._check_dev(actions, torch.uint8, (self.n,), "actions")
        if out is None:
            out = (self._u8(*self.obs_shape),
                   torch.empty(self.n, dtype=torch.float32, device=self.device),
                   self._u8(self.n))
        obs, rew, done = out
        self._check_dev(obs, torch.uint8, self.obs_shape, "obs")
        self._check_dev(rew, torch.float32, (self.n,), "reward")
        self._check_dev(done, torch.uint8, (self.n,), "done")
        check(load_library().octax_step(self._h, _ptr(actions), _ptr(obs), _ptr(rew), _ptr(done)))
        return obs, rew, done

    def step_n(self, actions, out=None):
        torch = self._torch
        T = int(actions.shape[0])
        self._check_dev(actions, torch.uint8, (T, self.n), "actions")
        if out is None:
            out = (self._u8(T, *self.obs_shape),
                   torch.empty((T, self.n), dtype=torch.float32, device=self.device),
                   self._u8(T, self.n))
        obs, rew, done = out
        self._check_dev(obs, torch.uint8, (T, *self.obs_shape), "obs")
        self._check_dev(rew, torch.float32, (T, self.n), "reward")
        self._check_dev(done, torch.uint8, (T, self.n), "done")
        check(load_library().octax_step_n(self._h, T, _ptr(actions), _ptr(obs), _ptr(rew),
                                          _ptr(done)))
        return obs, rew, done

    @property
    def packed_obs_shape(self) -> tuple:
        """Per-instance packed observation: (S, 32) CHIP-8 or (S, 128) SCHIP words."""
        return (self.S, 32 if self.frame == (32, 64) else 128)

    def step_n_packed(self, actions, out=None):
        """step_n with bit-packed observations: int64 words [T, n, S, W] (bit x of
        a word = pixel x of its 64-pixel run; see octax_step_n_packed)."""
        torch = self._torch
        T = int(actions.shape[0])
        self._check_dev(actions, torch.uint8, (T, self.n), "actions")
        if out is None:
            out = (torch.empty((T, self.n) + self.packed_obs_shape, dtype=torch.int64, device=self.device),
                   torch.empty((T, self.n), dtype=torch.float32, device=self.device),
                   self._u8(T, self.n))
        obs, rew, done = out
        self._check_dev(obs, torch.int64, (T, self.n) + self.packed_obs_shape, "obs")
        self._check_dev(rew, torch.float32, (T, self.n), "reward")
        self._check_dev(done, torch.uint8, (T, self.n), "done")
        check(load_library().octax_step_n_packed(self._h, T, _ptr(actions), _ptr(obs), _ptr(rew),
                                                 _ptr(done)))
        return obs, rew, done

    def step_host(self, actions, out=None):
        """Host buffers in and out (pinned CPU tensors copy fastest); synchronous."""
        torch = self._torch
        if out is None:
            out = (torch.empty(self.obs_shape, dtype=torch.uint8, pin_memory=True),
                   torch.empty(self.n, dtype=torch.float32, pin_memory=True),
                   torch.empty(self.n, dtype=torch.uint8, pin_memory=True))
        obs, rew, done = out
        for t, dt, shp, nm in ((actions, torch.uint8, (self.n,), "actions"),
                               (obs, torch.uint8, self.obs_shape, "obs"),
                               (rew, torch.float32, (self.n,), "reward"),
                               (done, torch.uint8, (self.n,), "done")):
            if t.device.type != "cpu" or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError(f"{nm}: need contiguous host {dt} {shp}")
        check(load_library().octax_step_host(self._h, _ptr(actions), _ptr(obs), _ptr(rew),
                                             _ptr(done)))
        return obs, rew, done

    def step_host_packed(self, actions, out=None):
        """step_host with packed frames (int64 words [n, S, W], see
        step_n_packed): 8x fewer observation bytes over the host link."""
        torch = self._torch
        if out is None:
            out = (torch.empty((self.n,) + self.packed_obs_shape, dtype=torch.int64, pin_memory=True),
                   torch.empty(self.n, dtype=torch.float32, pin_memory=True),
                   torch.empty(self.n, dtype=torch.uint8, pin_memory=True))
        obs, rew, done = out
        for t, dt, shp, nm in ((actions, torch.uint8, (self.n,), "actions"),
                               (obs, torch.int64, (self.n,) + self.packed_obs_shape, "obs"),
                               (rew, torch.float32, (self.n,), "reward"),
                               (done, torch.uint8, (self.n,), "done")):
            if t.device.type != "cpu" or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError(f"{nm}: need contiguous host {dt} {shp}")
        check(load_library().octax_step_host_packed(self._h, _ptr(actions), _ptr(obs), _ptr(rew),
                                                    _ptr(done)))
        return obs, rew, done

    def state_hash(self, out=None):
        torch = self._torch
        h = out if out is not None else torch.empty(self.n, dtype=torch.int64, device=self.device)
        self._check_dev(h, torch.int64, (self.n,), "hash")
        check(load_library().octax_state_hash(self._h, _ptr(h)))
        return h

    def get_state(self, first: int = 0, count: int | None = None) -> np.ndarray:
        count = self.n - first if count is None else count
        out = np.zeros(count, dtype=RECORD_DTYPE)
        check(load_library().octax_get_state(self._h, first, count, C.c_void_p(out.ctypes.data)))
        return out

    def set_state(self, records: np.ndarray, first: int = 0) -> None:
        rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
        check(load_library().octax_set_state(self._h, first, len(rec), C.c_void_p(rec.ctypes.data)))

    def sync(self, timeout_ms: int = -1) -> None:
        check(load_library().octax_sync(self._h, timeout_ms))

    def debug_stall_writers(self, on: bool) -> None:
        """Diagnostic: make the writer warps skip their hand-over so that the
        bounded waits of the warp-specialised kernel run out (see
        octax_debug_stall_writers)."""
        check(load_library().octax_debug_stall_writers(self._h, 1 if on else 0))

    @property
    def launch(self) -> dict:
        c = CLaunch()
        check(load_library().octax_get_launch(self._h, C.byref(c)))
        return {"block": c.block, "inst_per_warp": c.inst_per_warp,
                "steps_per_launch": c.steps_per_launch, "persistent": c.persistent,
                "use_graph": c.use_graph, "writer_warps": c.writer_warps, "balance": c.balance}

    def set_launch(self, **kw) -> None:
        cur = self.launch
        cur.update(kw)
        c = CLaunch(cur["block"], cur["inst_per_warp"], cur["steps_per_launch"], cur["persistent"],
                    cur["use_graph"], cur["writer_warps"], cur["balance"])
        check(load_library().octax_set_launch(self._h, C.byref(c)))

    def autotune(self, n_steps: int = 8, actions=None) -> float:
        """Pick the fastest launch configuration for step_n calls of n_steps
        steps (actions: representative uint8 [n_steps, n] device tensor)."""
        if actions is not None:
            self._check_dev(actions, self._torch.uint8, (n_steps, self.n), "actions")
        ms = C.c_float()
        check(load_library().octax_autotune(self._h, n_steps, _ptr(actions), C.byref(ms)))
        return ms.value

    @property
    def device_bytes(self) -> int:
        return int(load_library().octax_device_bytes(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load_library().octax_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (octax_server_*) on one GPU.

    ``submit`` queues a request for ``n_envs`` fresh instances of one game,
    stepped ``n_steps`` times with ``actions`` (uint8 [n_steps, n_envs]); the
    outputs land in device tensors that stay referenced here until the
    request is released."""

    def __init__(self, games, *, memory_budget_bytes: int, block: int = 64,
                 inst_per_warp: int = 8, max_inflight_ticks: int = 2, quirks: int = 0,
                 device=None):
        import torch

        self._torch = torch
        L = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.games = list(games)
        self.S = int(self.games[0].stack_frames)
        self.frame = frame_shape(getattr(self.games[0], "variant", "chip8"))
        keep = [make_game(g) for g in self.games]
        arr = (CGame * len(keep))(*[k[0] for k in keep])
        cfg = CServerConfig(int(memory_budget_bytes), block, inst_per_warp, max_inflight_ticks, 0)
        h = C.c_void_p()
        check(L.octax_server_create(arr, len(keep), quirks, C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = keep
        self._outs: dict[int, tuple] = {}

    def submit(self, game: int, actions: np.ndarray, seed: int, out=None) -> int:
        torch = self._torch
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        if a.ndim != 2:
            raise ValueError("actions: need uint8 [n_steps, n_envs]")
        T, n = a.shape
        if out is None:
            out = (torch.empty((T, n, self.S) + self.frame, dtype=torch.uint8, device=self.device),
                   torch.empty((T, n), dtype=torch.float32, device=self.device),
                   torch.empty((T, n), dtype=torch.uint8, device=self.device))
        obs, rew, done = out
        # the library sees plain pointers: the sizes are checked here
        for t, dt, shp, nm in ((obs, torch.uint8, (T, n, self.S) + self.frame, "obs"),
                               (rew, torch.float32, (T, n), "reward"),
                               (done, torch.uint8, (T, n), "done")):
            if t.device != self.device or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError(f"{nm}: need contiguous {dt} {shp} on {self.device}, "
                                 f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        req = CRequest(game, 0, n, T, 0, seed & 0xFFFFFFFFFFFFFFFF, a.ctypes.data,
                       obs.data_ptr(), rew.data_ptr(), done.data_ptr())
        rid = C.c_uint64()
        check(load_library().octax_server_submit(self._h, C.byref(req), C.byref(rid)))
        self._outs[rid.value] = out
        return rid.value

    def submit_batch(self, items) -> list:
        """Queue several requests at once: items = [(game, actions, seed, out)];
        out = (obs, reward, done) device tensors as in submit (required here)."""
        torch = self._torch
        arr = (CRequest * len(items))()
        keep = []
        for k, (game, actions, seed, out) in enumerate(items):
            a = np.ascontiguousarray(actions, dtype=np.uint8)
            T, n = a.shape
            obs, rew, done = out
            if obs.dtype != torch.uint8 or tuple(obs.shape) != (T, n, self.S) + self.frame or \
                    rew.dtype != torch.float32 or tuple(rew.shape) != (T, n) or \
                    done.dtype != torch.uint8 or tuple(done.shape) != (T, n) or \
                    not (obs.is_contiguous() and rew.is_contiguous() and done.is_contiguous()):
                raise ValueError("submit_batch: outputs must match each request's shape")
            keep.append(a)
            arr[k] = CRequest(game, 0, n, T, 0, seed & 0xFFFFFFFFFFFFFFFF, a.ctypes.data,
                              obs.data_ptr(), rew.data_ptr(), done.data_ptr())
        ids = (C.c_uint64 * len(items))()
        check(load_library().octax_server_submit_batch(self._h, arr, len(items), ids))
        out_ids = list(ids)
        for rid, it in zip(out_ids, items):
            self._outs[rid] = it[3]
        return out_ids

    REQUEST_DTYPE = np.dtype([("game", "<u2"), ("pad", "<u2"), ("n_envs", "<u4"), ("n_steps", "<u4"),
                              ("pad2", "<u4"), ("seed", "<u8"), ("actions", "<u8"), ("obs", "<u8"),
                              ("reward", "<u8"), ("done", "<u8")])

    def submit_raw(self, reqs: np.ndarray) -> np.ndarray:
        """Queue requests given as a REQUEST_DTYPE array (the octax_request
        layout: host action pointers, device output pointers, which the
        caller keeps alive until the requests are done). Returns the ids."""
        reqs = np.ascontiguousarray(reqs, dtype=self.REQUEST_DTYPE)
        assert self.REQUEST_DTYPE.itemsize == C.sizeof(CRequest)
        ids = np.zeros(len(reqs), dtype=np.uint64)
        check(load_library().octax_server_submit_batch(self._h, reqs.ctypes.data_as(C.POINTER(CRequest)),
                                                       len(reqs), ids.ctypes.data_as(C.POINTER(C.c_uint64))))
        return ids

    def wait_raw(self, ids: np.ndarray, release: bool = True, timeout_ms: int = -1) -> np.ndarray:
        """Wait for all ids; returns int64 [n, 3] (submit_ns, admit_ns, done_ns)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        infos = (CRequestInfo * len(ids))()
        check(load_library().octax_server_wait_batch(self._h, ids.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                     len(ids), timeout_ms, infos, int(release)))
        raw = np.frombuffer(infos, dtype=np.int64).reshape(len(ids), 4)
        return raw[:, 1:].copy()

    def wait_batch(self, ids, release: bool = True, timeout_ms: int = -1) -> list:
        """Wait for all ids; returns their infos; release=True forgets them."""
        arr = (C.c_uint64 * len(ids))(*ids)
        infos = (CRequestInfo * len(ids))()
        check(load_library().octax_server_wait_batch(self._h, arr, len(ids), timeout_ms, infos, int(release)))
        if release:
            for rid in ids:
                self._outs.pop(rid, None)
        return [self._info(i) for i in infos]

    def outputs(self, rid: int) -> tuple:
        return self._outs[rid]

    @staticmethod
    def _info(i: CRequestInfo) -> dict:
        return {"state": i.state, "submit_ns": i.submit_ns, "admit_ns": i.admit_ns,
                "done_ns": i.done_ns}

    def wait(self, rid: int, timeout_ms: int = -1) -> dict:
        info = CRequestInfo()
        check(load_library().octax_server_wait(self._h, rid, timeout_ms, C.byref(info)))
        return self._info(info)

    def query(self, rid: int) -> dict:
        info = CRequestInfo()
        check(load_library().octax_server_query(self._h, rid, C.byref(info)))
        return self._info(info)

    def release(self, rid: int) -> None:
        check(load_library().octax_server_release(self._h, rid))
        self._outs.pop(rid, None)

    def stats(self) -> dict:
        st = CServerStats()
        check(load_library().octax_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in CServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load_library().octax_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Policy:
    """The §4.1 actor-critic network on the tensor cores (octax_policy_*).

    params: dict of float32 arrays in the layouts of octax_policy_params
    (w1 [32,4,8,4], b1, w2 [64,32,4,4], b2, w3 [64,64,3,3], b3, wa1 / wc1
    [256,1024], ba1 / bc1, wa2 [L,256], ba2 [L], wc2 [256], bc2 [1])."""

    _NAMES = ("w1", "b1", "w2", "b2", "w3", "b3", "wa1", "ba1", "wa2", "ba2", "wc1", "bc1", "wc2", "bc2")

    def __init__(self, params: dict, max_envs: int, *, device=None, stream=None):
        import torch

        self._torch = torch
        L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("liboctax needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n_logits = int(np.asarray(params["wa2"]).shape[0])
        self.max_envs = int(max_envs)
        keep = {k: np.ascontiguousarray(params[k], dtype=np.float32) for k in self._NAMES}
        cp = CPolicyParams(*[C.c_void_p(keep[k].ctypes.data) for k in self._NAMES], self.n_logits)
        h = C.c_void_p()
        check(L.octax_policy_create(C.byref(cp), self.max_envs, self.device.index,
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def _outputs(self, n, out):
        torch = self._torch
        if out is None:
            out = (torch.empty((n, self.n_logits), dtype=torch.float32, device=self.device),
                   torch.empty(n, dtype=torch.float32, device=self.device),
                   torch.empty(n, dtype=torch.uint8, device=self.device))
        return out

    def forward(self, obs_words, seed: int = 0, step: int = 0, out=None):
        """Packed observations int64 [n, 4, 32] -> (logits [n, L], value [n], actions [n])."""
        torch = self._torch
        n = int(obs_words.shape[0])
        if obs_words.dtype != torch.int64 or tuple(obs_words.shape) != (n, 4, 32) or not obs_words.is_contiguous():
            raise ValueError("obs_words: need contiguous int64 [n, 4, 32]")
        lg, v, a = self._outputs(n, out)
        check(load_library().octax_policy_forward(self._h, n, _ptr(obs_words), seed & 0xFFFFFFFFFFFFFFFF,
                                                  step & 0xFFFFFFFF, _ptr(lg), _ptr(v), _ptr(a)))
        return lg, v, a

    def forward_u8(self, obs, seed: int = 0, step: int = 0, out=None):
        """uint8 observations [n, 4, 32, 64] -> (logits, value, actions)."""
        torch = self._torch
        n = int(obs.shape[0])
        if obs.dtype != torch.uint8 or tuple(obs.shape) != (n, 4, 32, 64) or not obs.is_contiguous():
            raise ValueError("obs: need contiguous uint8 [n, 4, 32, 64]")
        lg, v, a = self._outputs(n, out)
        check(load_library().octax_policy_forward_u8(self._h, n, _ptr(obs), seed & 0xFFFFFFFFFFFFFFFF,
                                                     step & 0xFFFFFFFF, _ptr(lg), _ptr(v), _ptr(a)))
        return lg, v, a

    def rollout(self, env: "Env", n_steps: int, obs_words, seed: int = 0, step0: int = 0, out=None,
                logits: bool = True):
        """octax_rollout_policy: n_steps on-device steps in which this policy
        acts. obs_words int64 [n, 4, 32] (updated in place to the last
        observation). Returns (actions [T,n], logits [T,n,L] or None,
        value [T,n], reward [T,n], done [T,n])."""
        torch = self._torch
        n, T = env.n, int(n_steps)
        if obs_words.dtype != torch.int64 or tuple(obs_words.shape) != (n, 4, 32) or not obs_words.is_contiguous():
            raise ValueError("obs_words: need contiguous int64 [n, 4, 32]")
        if out is None:
            out = (torch.empty((T, n), dtype=torch.uint8, device=self.device),
                   torch.empty((T, n, self.n_logits), dtype=torch.float32, device=self.device) if logits else None,
                   torch.empty((T, n), dtype=torch.float32, device=self.device),
                   torch.empty((T, n), dtype=torch.float32, device=self.device),
                   torch.empty((T, n), dtype=torch.uint8, device=self.device))
        a, lg, v, r, d = out
        check(load_library().octax_rollout_policy(env._h, self._h, T, seed & 0xFFFFFFFFFFFFFFFF,
                                                  step0 & 0xFFFFFFFF, _ptr(obs_words), _ptr(a), _ptr(lg),
                                                  _ptr(v), _ptr(r), _ptr(d)))
        return a, lg, v, r, d

    def sync(self) -> None:
        check(load_library().octax_policy_sync(self._h))

    def debug_stall(self, on: bool) -> None:
        """Diagnostic: make the conv kernel's first wait run out (octax_policy_debug_stall)."""
        check(load_library().octax_policy_debug_stall(self._h, int(bool(on))))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load_library().octax_policy_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
