"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/octax.h declares; the binding's struct layouts match the header."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"\b(octax_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_01764_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2510_01764_gb300 import octax

    assert set(octax.EXPORTS) <= set(declared_functions())


LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "octax.h"
#define P(T) printf(#T " %zu\n", sizeof(T))
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  P(octax_term); P(octax_clause); P(octax_game); P(octax_state_record); P(octax_launch);
  P(octax_server_config); P(octax_request); P(octax_request_info); P(octax_server_stats);
  O(octax_game, rom_len); O(octax_game, action_set); O(octax_game, score); O(octax_game, term);
  O(octax_game, max_episode_steps); O(octax_game, startup_instrs);
  O(octax_state_record, display); O(octax_state_record, ram); O(octax_state_record, env_steps);
  O(octax_request, seed); O(octax_request, actions_host); O(octax_request, done_dev);
  return 0;
}
"""


def test_struct_layouts_match_header(tmp_path):
    """Compile the header with gcc and compare every size/offset with ctypes."""
    import subprocess

    from paper_2510_01764_gb300 import octax as o

    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    sizes = {"octax_term": o.CTerm, "octax_clause": o.CClause, "octax_game": o.CGame,
             "octax_launch": o.CLaunch, "octax_server_config": o.CServerConfig,
             "octax_request": o.CRequest, "octax_request_info": o.CRequestInfo,
             "octax_server_stats": o.CServerStats}
    for name, cls in sizes.items():
        assert int(got[name]) == C.sizeof(cls), name
    assert int(got["octax_state_record"]) == o.RECORD_DTYPE.itemsize
    for key, val in got.items():
        if "." not in key:
            continue
        struct, field = key.split(".")
        if struct == "octax_state_record":
            assert int(val) == o.RECORD_DTYPE.fields[field][1], key
        else:
            cls = {"octax_game": o.CGame, "octax_request": o.CRequest}[struct]
            assert int(val) == getattr(cls, field).offset, key


def test_descriptor_validation_without_gpu(lib):
    """octax_create rejects bad descriptors before touching the device."""
    from paper_2510_01764_gb300 import octax as o
    from paper_2510_01764_gb300.workloads import GameSpec

    L = o.load_library()
    bad = [GameSpec(rom=b""), GameSpec(rom=b"\x00" * 3585), GameSpec(rom=b"\x12\x00", frameskip=2),
           GameSpec(rom=b"\x12\x00", instr_per_frame=0), GameSpec(rom=b"\x12\x00", action_set=(16,)),
           GameSpec(rom=b"\x12\x00", startup_instrs=(1 << 20) + 1),
           GameSpec(rom=b"\x12\x00", max_noops=256)]
    for g in bad:
        cg, keep = o.make_game(g) if len(g.rom) else (o.CGame(), None)
        arr = (o.CGame * 1)(cg)
        h = C.c_void_p()
        rc = L.octax_create(arr, 1, None, None, 4, 0, 0, None, C.byref(h))
        assert rc == o.EINVAL, g
        assert L.octax_last_error()
    cg, keep = o.make_game(GameSpec(rom=b"\x12\x00"))
    arr = (o.CGame * 1)(cg)
    h = C.c_void_p()
    assert L.octax_create(arr, 1, None, None, 0, 0, 0, None, C.byref(h)) == o.EINVAL
    assert L.octax_create(arr, 1, None, None, 4, 0x40, 0, None, C.byref(h)) == o.EINVAL
    assert L.octax_create(arr, 0, None, None, 4, 0, 0, None, C.byref(h)) == o.EINVAL


def test_binding_refuses_without_library(tmp_path):
    from paper_2510_01764_gb300 import octax

    saved = octax._lib
    octax._lib = None
    try:
        with pytest.raises(ImportError):
            octax.load_library(str(tmp_path / "missing.so"))
    finally:
        octax._lib = saved


def test_last_error_without_gpu(lib):
    lib.octax_last_error.restype = C.c_char_p
    assert isinstance(lib.octax_last_error(), bytes)
    lib.octax_num_envs.restype = C.c_int64
    lib.octax_num_envs.argtypes = [C.c_void_p]
    assert lib.octax_num_envs(None) == -1


def test_step_entry_points_reject_null_env_without_gpu(lib):
    """Every stepping / state entry point returns OCTAX_EINVAL with a message
    for a null environment, before touching the device."""
    from paper_2510_01764_gb300 import octax as o

    L = o.load_library()
    calls = {
        "octax_reset": (None, None, None),
        "octax_step": (None, None, None, None, None),
        "octax_step_n": (None, 1, None, None, None, None),
        "octax_step_n_packed": (None, 1, None, None, None, None),
        "octax_step_host": (None, None, None, None, None),
        "octax_step_host_packed": (None, None, None, None, None),
        "octax_state_hash": (None, None),
        "octax_get_state": (None, 0, 1, None),
        "octax_set_state": (None, 0, 1, None),
        "octax_sync": (None, 0),
    }
    for name, args in calls.items():
        fn = getattr(L, name)
        L.octax_last_error()
        assert fn(*args) == o.EINVAL, name
        assert name.encode() in L.octax_last_error(), name


def test_server_submit_checks_output_tensors_without_gpu():
    """The library takes plain device pointers, so the binding checks the
    output tensors' shape, dtype and device before a request is submitted."""
    import numpy as np

    torch = pytest.importorskip("torch")
    from paper_2510_01764_gb300 import octax as o

    srv = object.__new__(o.Server)          # no device needed: the check runs first
    srv._torch, srv.device, srv.S, srv.frame = torch, torch.device("cpu"), 4, (32, 64)
    T, n = 2, 8
    good = (torch.empty((T, n, 4, 32, 64), dtype=torch.uint8), torch.empty((T, n)),
            torch.empty((T, n), dtype=torch.uint8))
    bad = [(torch.empty((T, n, 4, 32, 63), dtype=torch.uint8),) + good[1:],
           (good[0], torch.empty((T, n), dtype=torch.float64), good[2]),
           good[:2] + (torch.empty((T + 1, n), dtype=torch.uint8),)]
    for out in bad:
        with pytest.raises(ValueError):
            srv.submit(0, np.zeros((T, n), np.uint8), 1, out=out)
    with pytest.raises(ValueError):
        srv.submit(0, np.zeros(n, np.uint8), 1, out=good)
