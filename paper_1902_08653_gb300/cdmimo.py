"""Python binding of the cdmimo C ABI (argument marshalling only).

Every function takes torch tensors as plain device (or pinned host) buffers, checks their dtype,
shape and contiguity, and passes raw pointers and the current CUDA stream to the C entry point of
the same name; all computation happens in the library's CUDA kernels.  There is no CPU fallback:
if libcdmimo.so is missing or fails to load, every call raises.

Tensor conventions (see include/cdmimo.h for the exact layouts):
  complex entries are torch.complex64, or 16-bit storage given as a [..., 2] tensor of
  torch.float16 / torch.bfloat16 (re, im pairs) with per-subcarrier float32 scales.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

OK = 0
ERR_INVALID_ARG = -1
ERR_BAD_PARTITION = -2
ERR_UNSUPPORTED = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_WORKSPACE = -6

DEV_TIMEOUT = 0x1
DEV_BAD_N0 = 0x2
DEV_BAD_LEARNED = 0x4
LEARNED_BLOCK_BYTES = 4 * 4 + 16 * 4 * 2 + 64 * 4 + 4 * 4 + 64 * 65 * 2 + 64 * 2

C64, C16F, C16BF = 0, 1, 2
FUSE = {"equal": 0, "colnorm": 1, "learned": 2}
FORM = {"auto": 0, "residual": 1, "gram": 2, "gram_tc": 3, "gram_tc_phased": 4, "gram_tc_umma": 5}
OP_DETECT, OP_PRECODE, OP_FRAME = 0, 1, 2


class CdmimoError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {status_string(status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("n_sc", ctypes.c_int), ("n_sym", ctypes.c_int), ("B", ctypes.c_int), ("U", ctypes.c_int),
                ("C", ctypes.c_int), ("cluster_size", ctypes.POINTER(ctypes.c_int)), ("K", ctypes.c_int),
                ("Ex", ctypes.c_float), ("fuse", ctypes.c_int), ("rho", ctypes.c_float), ("in_dtype", ctypes.c_int),
                ("h_scale", ctypes.c_void_p), ("y_scale", ctypes.c_void_p), ("learned", ctypes.c_void_p),
                ("form", ctypes.c_int)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("n_sc", ctypes.c_int), ("n_sym", ctypes.c_int), ("B", ctypes.c_int),
                ("U", ctypes.c_int), ("C", ctypes.c_int), ("K", ctypes.c_int), ("fuse", ctypes.c_int),
                ("Ex", ctypes.c_float), ("rho", ctypes.c_float), ("cluster_size", ctypes.POINTER(ctypes.c_int)),
                ("H", ctypes.c_void_p), ("V", ctypes.c_void_p), ("N0", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("threads", ctypes.c_int), ("group_bytes", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("n_items", ctypes.c_int), ("n_groups", ctypes.c_int),
                ("C_max", ctypes.c_int), ("smem_bytes", ctypes.c_uint), ("offsets", ctypes.c_uint * 9),
                ("table_bytes", ctypes.c_size_t)]


_lib = None


def lib():
    """Load libcdmimo.so (building it first if the sources are newer).  Raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.OUT
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libcdmimo.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(path)
        P, I, F, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        PP = ctypes.POINTER(Params)
        sig = {
            "cdmimo_detect": ([PP, P, P, P, P, P, P, P, S, P], I),
            "cdmimo_precode": ([PP, P, P, P, P, S, P], I),
            "cdmimo_fuse": ([I, I, I, I, P, P, I, P, P], I),
            "cdmimo_detect_host": ([PP, P, P, P, P, P, S, P], I),
            "cdmimo_precode_host": ([PP, P, P, P, P, S, P], I),
            "cdmimo_detect_precode_host": ([PP, P, P, P, P, P, P, I, P, S, P], I),
            "cdmimo_workspace_size": ([PP, I], S),
            "cdmimo_selected_form": ([PP, I, P], I),
            "cdmimo_detect_precode": ([PP, P, P, P, P, P, P, P, S, P], I),
            "cdmimo_host_workspace_size": ([PP, I], S),
            "cdmimo_status_string": ([I], ctypes.c_char_p),
            "cdmimo_device_status": ([I], I),
            "cdmimo_version": ([], I),
            "cdmimo_check_bounded_wait": ([ctypes.c_uint, P], I),
            "cdmimo_learned_param_count": ([I, I, I], S),
            "cdmimo_learned_pack": ([P, I, I, I, P, P], I),
            "cdmimo_learned_grad": ([PP, I, P, P, P, P, P, P, P, S, P], I),
            "cdmimo_learned_workspace_size": ([PP, I], S),
            "cdmimo_adam_step": ([P, P, P, P, I, F, F, F, F, I, P], I),
            "cdmimo_learned_grad_noalloc": ([PP, I, P, P, P, P, P, P, P], I),
            "cdmimo_batch_default_plan": ([ctypes.POINTER(BatchPlan)], None),
            "cdmimo_batch_build": ([ctypes.POINTER(BatchDesc), I, ctypes.POINTER(BatchPlan), P, S], I),
            "cdmimo_detect_batched": ([ctypes.POINTER(BatchPlan), P, P, P], I),
            "cdmimo_detect_batched_stats": ([ctypes.POINTER(BatchPlan), P, P, P, P], I),
            "cdmimo_umma_layout_probe": ([I, P, P, P, P], I),
            "cdmimo_umma_rate_probe": ([I, I, I, P, P], I),
            "cdmimo_synth_uplink": ([ctypes.c_ulonglong, I, I, I, I, I, P, P, P, P, P, P, P], I),
            "cdmimo_fusion_weights": ([PP, P, P, P, P], I),
            "cdmimo_pipe_probe_sink_floats": ([], S),
            "cdmimo_pipe_probe": ([I, I, P, S, ctypes.POINTER(ctypes.c_double), P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().cdmimo_status_string(int(status)).decode()


def device_status(clear: bool = False) -> int:
    return lib().cdmimo_device_status(1 if clear else 0)


def _check(fn, rc):
    if rc != OK:
        raise CdmimoError(fn, rc)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype_of(t: torch.Tensor) -> int:
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.float16 and t.shape[-1] == 2:
        return C16F
    if t.dtype == torch.bfloat16 and t.shape[-1] == 2:
        return C16BF
    raise TypeError(f"unsupported storage {t.dtype} {tuple(t.shape)}: use complex64 or [...,2] float16/bfloat16")


def _need(t, name, dev=True):
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dev and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not dev and t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    return t


def make_params(n_sc, n_sym, B, U, cluster_size, K, *, Ex=1.0, fuse="colnorm", rho=1.0, in_dtype=C64,
                h_scale=None, y_scale=None, learned=None, form="auto"):
    """Build the C parameter block.  Returns (Params, keepalive) — keep both alive during the call."""
    cs = (ctypes.c_int * len(cluster_size))(*[int(v) for v in cluster_size])
    p = Params(int(n_sc), int(n_sym), int(B), int(U), len(cluster_size), ctypes.cast(cs, ctypes.POINTER(ctypes.c_int)),
               int(K), float(Ex), FUSE[fuse] if isinstance(fuse, str) else int(fuse), float(rho), int(in_dtype),
               h_scale.data_ptr() if h_scale is not None else None,
               y_scale.data_ptr() if y_scale is not None else None,
               learned.data_ptr() if learned is not None else None,
               FORM[form] if isinstance(form, str) else int(form))
    return p, cs


_PARAMS = {}


def _params_cached(*key):
    """make_params for the hot-path calls, memoized on every field (the parameter block is read by
    the library during the call only, so one block per distinct argument set can be reused)."""
    hit = _PARAMS.get(key)
    if hit is None:
        if len(_PARAMS) > 256:
            _PARAMS.clear()
        (n_sc, n_sym, B, U, cs, K, Ex, fuse, rho, in_dtype, hs, ys, learned, form) = key
        c = (ctypes.c_int * len(cs))(*cs)
        p = Params(n_sc, n_sym, B, U, len(cs), ctypes.cast(c, ctypes.POINTER(ctypes.c_int)), K, Ex,
                   FUSE[fuse] if isinstance(fuse, str) else int(fuse), rho, in_dtype, hs, ys, learned,
                   FORM[form] if isinstance(form, str) else int(form))
        hit = _PARAMS[key] = (ctypes.byref(p), p, c)
    return hit[0]


_SCHED = {}


def schedule_workspace(device, stream=None):
    """The zero-filled 256-byte schedule workspace this binding passes to cdmimo_detect /
    cdmimo_precode on (device, stream): one per stream, so calls on different streams never share
    counters (what workspace=True selects)."""
    device = torch.device(device)
    idx = device.index if device.index is not None else torch.cuda.current_device()
    return _sched_for(idx, _stream(stream).value, device)


def _sched_for(idx, stream_value, device):
    key = (idx, stream_value)
    ws = _SCHED.get(key)
    if ws is None:
        ws = _SCHED[key] = torch.zeros(int(lib().cdmimo_workspace_size(None, OP_DETECT)), dtype=torch.uint8,
                                       device=device)
    return ws


def _workspace_args(workspace, device, st):
    if workspace is None or workspace is False:
        return None, 0
    if workspace is True:
        workspace = _sched_for(device.index, st.value, device)
    return workspace.data_ptr(), workspace.numel() * workspace.element_size()


def _dptr(t):
    return t.data_ptr() if t is not None else None


def detect(H, Y, N0, cluster_size, K, *, Ex=1.0, fuse="colnorm", h_scale=None, y_scale=None, learned=None,
           out=None, Xc=None, lam=None, workspace=None, stream=None, form="auto"):
    """cdmimo_detect: Algorithm 1 + fusion.  Returns Xhat [n_sc, n_sym, U] complex64.
    workspace: None or False = static subcarrier schedule; True = dynamic schedule on this binding's
    per-stream counters; or a zero-filled device tensor of cdmimo_workspace_size bytes (dynamic).  form: "auto", "residual", "gram" or "gram_tc"
    (cdmimo_form)."""
    _need(H, "H")
    _need(Y, "Y")
    _need(N0, "N0")
    dt = _dtype_of(H)
    if _dtype_of(Y) != dt:
        raise TypeError("H and Y must use the same storage dtype")
    n_sc, U, B = H.shape[:3]
    n_sym = Y.shape[1]
    if N0.dtype != torch.float32:
        raise TypeError("N0 must be float32")
    if out is None:
        out = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=H.device)
    _need(out, "out")
    st = _stream(stream)
    pp = _params_cached(int(n_sc), int(n_sym), int(B), int(U), tuple(int(v) for v in cluster_size), int(K), float(Ex),
                        fuse, 1.0, dt, _dptr(h_scale), _dptr(y_scale), _dptr(learned), form)
    ws, wsb = _workspace_args(workspace, H.device, st)
    rc = lib().cdmimo_detect(pp, _ptr(H), _ptr(Y), _ptr(N0), _ptr(out), _ptr(Xc), _ptr(lam), ws, wsb, st)
    _check("cdmimo_detect", rc)
    return out


def precode(H, S, cluster_size, K, *, rho=1.0, out=None, workspace=None, stream=None, form="auto"):
    """cdmimo_precode: Algorithm 2 + per-cluster normalization.  Returns Xdl [n_sc, n_sym, B] complex64.
    workspace as for detect."""
    _need(H, "H")
    _need(S, "S")
    dt = _dtype_of(H)
    if S.dtype != torch.complex64:
        raise TypeError("S must be complex64")
    n_sc, U, B = H.shape[:3]
    n_sym = S.shape[1]
    if out is None:
        out = torch.empty((n_sc, n_sym, B), dtype=torch.complex64, device=H.device)
    _need(out, "out")
    st = _stream(stream)
    pp = _params_cached(int(n_sc), int(n_sym), int(B), int(U), tuple(int(v) for v in cluster_size), int(K), 1.0,
                        "colnorm", float(rho), dt, None, None, None, form)
    ws, wsb = _workspace_args(workspace, H.device, st)
    rc = lib().cdmimo_precode(pp, _ptr(H), _ptr(S), _ptr(out), ws, wsb, st)
    _check("cdmimo_precode", rc)
    return out


def detect_precode(H, Y, N0, S, cluster_size, K, *, Ex=1.0, fuse="colnorm", rho=1.0, h_scale=None, y_scale=None,
                   out=None, out_dl=None, workspace=None, stream=None, form="auto"):
    """cdmimo_detect_precode: one TDD frame on channel H (uplink detection of Y, downlink precoding
    of S).  Returns (Xhat [n_sc, n_sym, U], Xdl [n_sc, n_sym, B]) complex64."""
    _need(H, "H")
    _need(Y, "Y")
    _need(N0, "N0")
    _need(S, "S")
    dt = _dtype_of(H)
    if _dtype_of(Y) != dt:
        raise TypeError("H and Y must use the same storage dtype")
    if S.dtype != torch.complex64 or N0.dtype != torch.float32:
        raise TypeError("S must be complex64 and N0 float32")
    n_sc, U, B = H.shape[:3]
    n_sym = Y.shape[1]
    if out is None:
        out = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=H.device)
    if out_dl is None:
        out_dl = torch.empty((n_sc, n_sym, B), dtype=torch.complex64, device=H.device)
    _need(out, "out")
    _need(out_dl, "out_dl")
    st = _stream(stream)
    pp = _params_cached(int(n_sc), int(n_sym), int(B), int(U), tuple(int(v) for v in cluster_size), int(K), float(Ex),
                        fuse, float(rho), dt, _dptr(h_scale), _dptr(y_scale), None, form)
    ws, wsb = _workspace_args(workspace, H.device, st)
    rc = lib().cdmimo_detect_precode(pp, _ptr(H), _ptr(Y), _ptr(N0), _ptr(out), _ptr(S), _ptr(out_dl), ws, wsb, st)
    _check("cdmimo_detect_precode", rc)
    return out, out_dl


def fuse(Xc, w, *, weights_are_lambda=False, out=None, stream=None):
    """cdmimo_fuse: Xhat = sum_c lambda_c Xc[:, c] with lambda given, or derived from sigma_c^2."""
    _need(Xc, "Xc")
    _need(w, "w")
    n_sc, C, n_sym, U = Xc.shape
    if out is None:
        out = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=Xc.device)
    rc = lib().cdmimo_fuse(n_sc, n_sym, U, C, _ptr(Xc), _ptr(w), 1 if weights_are_lambda else 0, _ptr(out),
                           _stream(stream))
    _check("cdmimo_fuse", rc)
    return out


def selected_form(op, n_sc, n_sym, B, U, cluster_size, K, *, in_dtype=C64, form="auto", H=None):
    """cdmimo_selected_form: "residual", "gram" or (op OP_FRAME) "gram_tc", the form a call with these
    arguments runs."""
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, in_dtype=in_dtype, form=form)
    rc = lib().cdmimo_selected_form(ctypes.byref(p), op, _ptr(H) if H is not None else ctypes.c_void_p(256))
    if rc < 0:
        raise CdmimoError("cdmimo_selected_form", rc)
    return {v: k for k, v in FORM.items()}[rc]


def host_workspace_size(op, n_sc, n_sym, B, U, cluster_size, K, in_dtype=C64):
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, in_dtype=in_dtype)
    return int(lib().cdmimo_host_workspace_size(ctypes.byref(p), op))


def detect_host(H, Y, N0, cluster_size, K, Xhat, dev_ws, *, Ex=1.0, fuse="colnorm", h_scale=None, y_scale=None,
                stream=None):
    """cdmimo_detect_host: host (pinned) inputs and output; the copies are enqueued with the kernel.
    The caller synchronizes the stream before reading Xhat."""
    for t, nm in ((H, "H"), (Y, "Y"), (N0, "N0"), (Xhat, "Xhat")):
        _need(t, nm, dev=False)
    _need(dev_ws, "dev_ws")
    dt = _dtype_of(H)
    n_sc, U, B = H.shape[:3]
    n_sym = Y.shape[1]
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, Ex=Ex, fuse=fuse, in_dtype=dt, h_scale=h_scale,
                          y_scale=y_scale)
    rc = lib().cdmimo_detect_host(ctypes.byref(p), _ptr(H), _ptr(Y), _ptr(N0), _ptr(Xhat), _ptr(dev_ws),
                                  dev_ws.numel() * dev_ws.element_size(), _stream(stream))
    _check("cdmimo_detect_host", rc)
    return Xhat


def detect_precode_host(H, Y, N0, S, cluster_size, K, Xhat, Xdl, dev_ws, *, Ex=1.0, fuse="colnorm", rho=1.0,
                        h_scale=None, y_scale=None, n_chunks=0, stream=None, form="auto"):
    """cdmimo_detect_precode_host: one TDD frame on host (pinned) buffers, pipelined over n_chunks
    chunks of subcarriers (0: the library's default; 1: no pipelining).  dev_ws: device bytes of
    host_workspace_size(OP_FRAME, ...).  The caller synchronizes `stream` before reading Xhat, Xdl."""
    for t, nm in ((H, "H"), (Y, "Y"), (N0, "N0"), (S, "S"), (Xhat, "Xhat"), (Xdl, "Xdl")):
        _need(t, nm, dev=False)
    _need(dev_ws, "dev_ws")
    dt = _dtype_of(H)
    n_sc, U, B = H.shape[:3]
    n_sym = Y.shape[1]
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, Ex=Ex, fuse=fuse, rho=rho, in_dtype=dt,
                          h_scale=h_scale, y_scale=y_scale, form=form)
    rc = lib().cdmimo_detect_precode_host(ctypes.byref(p), _ptr(H), _ptr(Y), _ptr(N0), _ptr(S), _ptr(Xhat), _ptr(Xdl),
                                          int(n_chunks), _ptr(dev_ws), dev_ws.numel() * dev_ws.element_size(),
                                          _stream(stream))
    _check("cdmimo_detect_precode_host", rc)
    return Xhat, Xdl


def precode_host(H, S, cluster_size, K, Xdl, dev_ws, *, rho=1.0, stream=None):
    """cdmimo_precode_host: host (pinned) inputs and output."""
    for t, nm in ((H, "H"), (S, "S"), (Xdl, "Xdl")):
        _need(t, nm, dev=False)
    _need(dev_ws, "dev_ws")
    dt = _dtype_of(H)
    n_sc, U, B = H.shape[:3]
    n_sym = S.shape[1]
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, rho=rho, in_dtype=dt)
    rc = lib().cdmimo_precode_host(ctypes.byref(p), _ptr(H), _ptr(S), _ptr(Xdl), _ptr(dev_ws),
                                   dev_ws.numel() * dev_ws.element_size(), _stream(stream))
    _check("cdmimo_precode_host", rc)
    return Xdl


# ------------------------------------------------------------------------------------------------
# learned deep-unfolded CD
# ------------------------------------------------------------------------------------------------
def learned_param_count(K, U, hidden):
    return int(lib().cdmimo_learned_param_count(int(K), int(U), int(hidden)))


def learned_pack(master, K, U, hidden, block, stream=None):
    """cdmimo_learned_pack: masters (device float32) -> inference block (device, LEARNED_BLOCK_BYTES)."""
    _need(master, "master")
    _need(block, "block")
    if master.dtype != torch.float32 or master.numel() != learned_param_count(K, U, hidden):
        raise ValueError("master must be float32 of cdmimo_learned_param_count(K, U, hidden) entries")
    if block.numel() * block.element_size() < LEARNED_BLOCK_BYTES:
        raise ValueError("block too small")
    _check("cdmimo_learned_pack", lib().cdmimo_learned_pack(_ptr(master), int(K), int(U), int(hidden), _ptr(block),
                                                            _stream(stream)))
    return block


def learned_workspace_size(n_sc, n_sym, B, U, cluster_size, K, hidden):
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K)
    return int(lib().cdmimo_learned_workspace_size(ctypes.byref(p), int(hidden)))


def learned_grad(H, Y, N0, Xtarget, cluster_size, K, block, hidden, *, grad=None, loss=None, workspace=None,
                 Ex=1.0, stream=None):
    """cdmimo_learned_grad: loss and gradient w.r.t. the master parameters.  Returns (loss[1], grad)."""
    for t, nm in ((H, "H"), (Y, "Y"), (N0, "N0"), (Xtarget, "Xtarget"), (block, "block")):
        _need(t, nm)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    n = learned_param_count(K, U, hidden)
    if grad is None:
        grad = torch.empty(n, dtype=torch.float32, device=H.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=H.device)
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, Ex=Ex, fuse="learned", learned=block)
    need = int(lib().cdmimo_learned_workspace_size(ctypes.byref(p), int(hidden)))
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=H.device)
    rc = lib().cdmimo_learned_grad(ctypes.byref(p), int(hidden), _ptr(H), _ptr(Y), _ptr(N0), _ptr(Xtarget),
                                   _ptr(grad), _ptr(loss), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream))
    _check("cdmimo_learned_grad", rc)
    return loss, grad


def learned_grad_noalloc(H, Y, N0, Xtarget, cluster_size, K, block, hidden, *, grad, loss, Ex=1.0, stream=None):
    """cdmimo_learned_grad_noalloc: like learned_grad, with the library's fixed scratch instead of a
    caller workspace (for callers that cannot allocate device memory); grad and loss must be given."""
    for t, nm in ((H, "H"), (Y, "Y"), (N0, "N0"), (Xtarget, "Xtarget"), (block, "block"), (grad, "grad"),
                  (loss, "loss")):
        _need(t, nm)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    p, keep = make_params(n_sc, n_sym, B, U, cluster_size, K, Ex=Ex, fuse="learned", learned=block)
    rc = lib().cdmimo_learned_grad_noalloc(ctypes.byref(p), int(hidden), _ptr(H), _ptr(Y), _ptr(N0), _ptr(Xtarget),
                                           _ptr(grad), _ptr(loss), _stream(stream))
    _check("cdmimo_learned_grad_noalloc", rc)
    return loss, grad


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """cdmimo_adam_step on float32 device tensors (in place)."""
    for t, nm in ((theta, "theta"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t, nm)
    _check("cdmimo_adam_step", lib().cdmimo_adam_step(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(),
                                                      float(lr), float(beta1), float(beta2), float(eps), int(step),
                                                      _stream(stream)))


def synth_uplink(seed, n_sc, n_sym, B, U, snr_db, M=16, device="cuda", labels=False, stream=None):
    """cdmimo_synth_uplink: seeded synthetic uplink batch on the device.  snr_db: device float32 [n_sc].
    Returns dict(H, X, Y, N0[, labels])."""
    dev = torch.device(device)
    out = {"H": torch.empty((n_sc, U, B), dtype=torch.complex64, device=dev),
           "X": torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=dev),
           "Y": torch.empty((n_sc, n_sym, B), dtype=torch.complex64, device=dev),
           "N0": torch.empty(n_sc, dtype=torch.float32, device=dev)}
    lab = torch.empty((n_sc, n_sym, U), dtype=torch.int32, device=dev) if labels else None
    _need(snr_db, "snr_db")
    rc = lib().cdmimo_synth_uplink(int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_sc), int(n_sym), int(B), int(U), int(M),
                                   _ptr(snr_db), _ptr(out["H"]), _ptr(out["X"]), _ptr(lab), _ptr(out["Y"]),
                                   _ptr(out["N0"]), _stream(stream))
    _check("cdmimo_synth_uplink", rc)
    if labels:
        out["labels"] = lab
    return out


def check_bounded_wait(timeout_us=20000, stream=None):
    """cdmimo_check_bounded_wait: one thread's bounded wait on a barrier nothing completes expires
    after timeout_us and sets DEV_TIMEOUT (read it with device_status)."""
    _check("cdmimo_check_bounded_wait", lib().cdmimo_check_bounded_wait(int(timeout_us), _stream(stream)))


PROBE_FFMA2, PROBE_MMA_TF32 = 0, 1


def pipe_probe(kind, iters, sink, stream=None):
    """cdmimo_pipe_probe: enqueue one pipe-throughput probe launch; returns its flop count.  sink: a
    float32 device tensor of at least cdmimo_pipe_probe_sink_floats() elements."""
    _need(sink, "sink")
    fl = ctypes.c_double(0.0)
    _check("cdmimo_pipe_probe", lib().cdmimo_pipe_probe(int(kind), int(iters), _ptr(sink), sink.numel(),
                                                        ctypes.byref(fl), _stream(stream)))
    return fl.value


def pipe_probe_sink_floats():
    return int(lib().cdmimo_pipe_probe_sink_floats())


def umma_layout_probe(M, A, B, stream=None):
    """cdmimo_umma_layout_probe: D = A B^T on the tcgen05 tensor cores (A [M, 32], B [32, 32] float32
    device tensors, M 64 or 128); returns all 128 tensor-memory lanes x 32 columns as a [128, 32]
    tensor (lane-major)."""
    _need(A, "A")
    _need(B, "B")
    D = torch.full((128, 32), float("nan"), dtype=torch.float32, device=A.device)
    _check("cdmimo_umma_layout_probe", lib().cdmimo_umma_layout_probe(int(M), _ptr(A), _ptr(B), _ptr(D),
                                                                      _stream(stream)))
    return D


def umma_rate_probe(M, N, n, stream=None):
    """cdmimo_umma_rate_probe: SM cycles of n back-to-back M x N x 8 tf32 tcgen05 MMAs from one thread
    (best of five, commit and wait included); -1 if a wait timed out."""
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check("cdmimo_umma_rate_probe", lib().cdmimo_umma_rate_probe(int(M), int(N), int(n), _ptr(out),
                                                                  _stream(stream)))
    return int(out.item())


def fusion_weights(H, N0, cluster_size, *, Ex=1.0, fuse="colnorm", h_scale=None, out=None, stream=None):
    """cdmimo_fusion_weights: unnormalized Sec. III fusion weights [n_sc, C] (float32, device) of the
    clusters of H, in H's true units: the weights of cluster sets held by separate calls or devices
    concatenate, and lambda is their normalization over all clusters."""
    _need(H, "H")
    _need(N0, "N0")
    dt = _dtype_of(H)
    n_sc, U, B = H.shape[0], H.shape[1], H.shape[2]
    C = len(cluster_size)
    if out is None:
        out = torch.empty((n_sc, C), dtype=torch.float32, device=H.device)
    p, keep = make_params(n_sc, 1, B, U, cluster_size, 1, Ex=Ex, fuse=fuse, in_dtype=dt, h_scale=h_scale)
    _check("cdmimo_fusion_weights", lib().cdmimo_fusion_weights(ctypes.byref(p), _ptr(H), _ptr(N0), _ptr(out),
                                                                _stream(stream)))
    return out

