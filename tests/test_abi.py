"""The C-ABI library loads, exports every declared entry point, and validates arguments on the
host (CPU only: no call here reaches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_1902_08653_gb300 import cdmimo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cdmimo_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cdmimo_detect", "cdmimo_precode", "cdmimo_fuse", "cdmimo_workspace_size",
                     "cdmimo_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = cdmimo.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_version():
    for code, name in [(0, "CDMIMO_OK"), (-1, "CDMIMO_ERR_INVALID_ARG"), (-2, "CDMIMO_ERR_BAD_PARTITION"),
                       (-3, "CDMIMO_ERR_UNSUPPORTED"), (-4, "CDMIMO_ERR_CUDA"), (-5, "CDMIMO_ERR_TIMEOUT"),
                       (-6, "CDMIMO_ERR_WORKSPACE")]:
        assert cdmimo.status_string(code) == name
    assert cdmimo.status_string(12345) == "CDMIMO_UNKNOWN_STATUS"
    assert cdmimo.lib().cdmimo_version() >= 0x000100


def _detect_rc(**kw):
    args = dict(n_sc=4, n_sym=2, B=32, U=4, cluster_size=[16, 16], K=3)
    args.update(kw)
    p, keep = cdmimo.make_params(args["n_sc"], args["n_sym"], args["B"], args["U"], args["cluster_size"], args["K"],
                                 Ex=args.get("Ex", 1.0), fuse=args.get("fuse", "colnorm"),
                                 in_dtype=args.get("in_dtype", 0))
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: validation fails before any launch
    ptrs = [args.get(k, fake) for k in ("H", "Y", "N0", "Xhat")]
    return cdmimo.lib().cdmimo_detect(ctypes.byref(p), *ptrs, None, None, None, 0, None)


@pytest.mark.parametrize("kw,code", [
    (dict(cluster_size=[16, 15]), cdmimo.ERR_BAD_PARTITION),
    (dict(cluster_size=[32, 0]), cdmimo.ERR_BAD_PARTITION),
    (dict(cluster_size=[40, -8]), cdmimo.ERR_BAD_PARTITION),
    (dict(K=-1), cdmimo.ERR_INVALID_ARG),
    (dict(n_sym=0), cdmimo.ERR_INVALID_ARG),
    (dict(n_sc=-1), cdmimo.ERR_INVALID_ARG),
    (dict(U=0), cdmimo.ERR_INVALID_ARG),
    (dict(U=65), cdmimo.ERR_UNSUPPORTED),
    (dict(Ex=0.0), cdmimo.ERR_INVALID_ARG),
    (dict(Ex=float("nan")), cdmimo.ERR_INVALID_ARG),
    (dict(fuse=7), cdmimo.ERR_INVALID_ARG),
    (dict(in_dtype=9), cdmimo.ERR_INVALID_ARG),
    (dict(H=None), cdmimo.ERR_INVALID_ARG),
    (dict(Xhat=None), cdmimo.ERR_INVALID_ARG),
    (dict(Y=ctypes.c_void_p(0x10004)), cdmimo.ERR_INVALID_ARG),   # misaligned complex64
    (dict(in_dtype=1), cdmimo.ERR_INVALID_ARG),                   # 16-bit storage without scales
])
def test_detect_validation(kw, code):
    assert _detect_rc(**kw) == code


def test_empty_batch_is_a_no_op():
    assert _detect_rc(n_sc=0, H=None, Y=None, N0=None, Xhat=None) == cdmimo.OK


def test_precode_and_fuse_validation():
    L = cdmimo.lib()
    p, keep = cdmimo.make_params(2, 1, 32, 4, [16, 17], 3)
    fake = ctypes.c_void_p(0x10000)
    assert L.cdmimo_precode(ctypes.byref(p), fake, fake, fake, None, 0, None) == cdmimo.ERR_BAD_PARTITION
    p, keep = cdmimo.make_params(2, 1, 32, 4, [16, 16], 3)
    assert L.cdmimo_precode(ctypes.byref(p), None, fake, fake, None, 0, None) == cdmimo.ERR_INVALID_ARG
    assert L.cdmimo_fuse(2, 1, 4, 0, fake, fake, 0, fake, None) == cdmimo.ERR_INVALID_ARG
    assert L.cdmimo_fuse(2, 1, 4, 2, None, fake, 0, fake, None) == cdmimo.ERR_INVALID_ARG
    assert L.cdmimo_fuse(0, 1, 4, 2, None, None, 0, None, None) == cdmimo.OK


def test_host_workspace_sizes():
    L = cdmimo.lib()
    p, keep = cdmimo.make_params(1200, 14, 256, 16, [32] * 8, 3)
    need = L.cdmimo_host_workspace_size(ctypes.byref(p), cdmimo.OP_DETECT)
    assert need >= 1200 * 16 * 256 * 8 + 1200 * 14 * 256 * 8 + 1200 * 4 + 1200 * 14 * 16 * 8
    assert need % 256 == 0
    assert L.cdmimo_workspace_size(ctypes.byref(p), cdmimo.OP_DETECT) == 256
    assert L.cdmimo_workspace_size(ctypes.byref(p), cdmimo.OP_PRECODE) == 256
    assert L.cdmimo_detect_host(ctypes.byref(p), ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                ctypes.c_void_p(1), ctypes.c_void_p(256), 16, None) == cdmimo.ERR_WORKSPACE


def test_frame_host_workspace_and_validation():
    L = cdmimo.lib()
    n, ns, B, U = 1200, 14, 256, 16
    p, keep = cdmimo.make_params(n, ns, B, U, [32] * 8, 3)
    r = lambda v: (v + 255) // 256 * 256
    need = L.cdmimo_host_workspace_size(ctypes.byref(p), cdmimo.OP_FRAME)
    # staging of H, Y, N0, S, Xhat and Xdl, each 256-byte aligned (no schedule counters: static schedule)
    assert need == r(n * U * B * 8) + r(n * ns * B * 8) + r(n * 4) + 2 * r(n * ns * U * 8) + r(n * ns * B * 8)
    q, keep2 = cdmimo.make_params(n, ns, B, U, [32] * 8, 3, in_dtype=cdmimo.C16BF, h_scale=None, y_scale=None)
    assert L.cdmimo_host_workspace_size(ctypes.byref(q), cdmimo.OP_FRAME) == \
        r(n * U * B * 4) + r(n * ns * B * 4) + 3 * r(n * 4) + 2 * r(n * ns * U * 8) + r(n * ns * B * 8)
    assert L.cdmimo_host_workspace_size(ctypes.byref(p), 3) == 0
    one = ctypes.c_void_p(256)
    args = [one] * 6
    call = lambda a, chunks=0, ws=one, wsb=need: L.cdmimo_detect_precode_host(ctypes.byref(p), *a, chunks, ws, wsb,
                                                                             None)
    assert call(args[:2] + [None] + args[3:]) == cdmimo.ERR_INVALID_ARG  # no N0
    assert call(args[:5] + [None]) == cdmimo.ERR_INVALID_ARG  # no Xdl
    assert call(args, chunks=-1) == cdmimo.ERR_INVALID_ARG
    assert call(args, ws=None) == cdmimo.ERR_WORKSPACE
    assert call(args, wsb=need - 1) == cdmimo.ERR_WORKSPACE
    assert call(args, ws=ctypes.c_void_p(256 + 16)) == cdmimo.ERR_WORKSPACE  # not 256-byte aligned
    assert call(args, ws=None, chunks=-1) == cdmimo.ERR_INVALID_ARG
    e, keep3 = cdmimo.make_params(0, ns, B, U, [32] * 8, 3)
    assert L.cdmimo_detect_precode_host(ctypes.byref(e), *([None] * 6), 0, None, 0, None) == cdmimo.OK


def test_form_validation_and_query():
    L = cdmimo.lib()
    p, keep = cdmimo.make_params(8, 14, 256, 16, [32] * 8, 3, form=7)
    one = ctypes.c_void_p(256)
    assert L.cdmimo_detect(ctypes.byref(p), one, one, one, one, None, None, None, 0, None) == cdmimo.ERR_INVALID_ARG
    assert L.cdmimo_selected_form(ctypes.byref(p), cdmimo.OP_DETECT, one) == cdmimo.ERR_INVALID_ARG
    p, keep = cdmimo.make_params(8, 14, 256, 16, [32] * 8, 3, form="residual")
    assert L.cdmimo_selected_form(ctypes.byref(p), cdmimo.OP_DETECT, one) == cdmimo.FORM["residual"]
    assert L.cdmimo_selected_form(ctypes.byref(p), 9, one) == cdmimo.ERR_INVALID_ARG


def test_schedule_workspace_validation():
    # misaligned or short schedule workspaces are rejected before anything touches the device
    L = cdmimo.lib()
    p, keep = cdmimo.make_params(8, 14, 256, 16, [32] * 8, 3)
    one = ctypes.c_void_p(256)
    for ws, nb in ((ctypes.c_void_p(8), 256), (ctypes.c_void_p(4096), 255)):
        assert L.cdmimo_detect(ctypes.byref(p), one, one, one, one, None, None, ws, nb, None) == cdmimo.ERR_WORKSPACE
        assert L.cdmimo_precode(ctypes.byref(p), one, one, one, ws, nb, None) == cdmimo.ERR_WORKSPACE


def test_learned_block_layout_and_param_count():
    class Block(ctypes.Structure):
        _fields_ = [("K", ctypes.c_int), ("U", ctypes.c_int), ("hidden", ctypes.c_int), ("r0", ctypes.c_int),
                    ("tau", ctypes.c_float * 16), ("gamma", ctypes.c_float * 16), ("b1", ctypes.c_float * 64),
                    ("b2", ctypes.c_float), ("r1", ctypes.c_float * 3), ("W1", ctypes.c_uint16 * (64 * 65)),
                    ("w2", ctypes.c_uint16 * 64)]

    assert ctypes.sizeof(Block) == cdmimo.LEARNED_BLOCK_BYTES
    assert cdmimo.learned_param_count(2, 16, 64) == 2 * 2 + 64 * 17 + 2 * 64 + 1
    assert cdmimo.learned_param_count(0, 16, 64) == 0
    assert cdmimo.learned_param_count(17, 16, 64) == 0
    assert cdmimo.learned_param_count(2, 16, 65) == 0
    L = cdmimo.lib()
    assert L.cdmimo_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == cdmimo.ERR_INVALID_ARG
    assert L.cdmimo_learned_pack(None, 2, 16, 64, None, None) == cdmimo.ERR_INVALID_ARG


def test_check_bounded_wait_rejects_limits_out_of_range():
    L = cdmimo.lib()
    for us in (0, 2000001, 4000000000):
        assert L.cdmimo_check_bounded_wait(us, None) == cdmimo.ERR_INVALID_ARG
