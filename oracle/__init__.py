"""FP64 CPU oracle for decentralized CD detection and precoding (arXiv 1902.08653).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The product (the CUDA library and its Python binding) never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``cdmimo_oracle.c`` (plain C99, double precision); this module only builds
it with gcc, loads it with ctypes and marshals numpy arrays.  ctypes releases the GIL during a
call, so ``threads > 1`` splits the subcarriers over a thread pool.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` and
``tests/test_oracle_learned.py`` (closed forms, library solves, matrix-splitting forms, invariants,
brute force; the learned fusion by hand-set weights whose logits are derived by hand), except the fusion-weight rule
for ``fuse="colnorm"``, whose formula is a reading of an under-specified passage (Sec. III): it is
pinned only by its invariants (weights sum to one, equal clusters get equal weights, a scaled
cluster gets the closed-form weight), not by a value the paper prints.
"""
from __future__ import annotations

import concurrent.futures as _fut
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdmimo_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libcdmimo_oracle.so")
_lib = None

FUSE = {"equal": 0, "colnorm": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE double; no fast-math)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        P = ctypes.c_void_p
        i = ctypes.c_int
        d = ctypes.c_double
        L.oracle_detect.argtypes = [i, i, i, i, i, P, i, d, i, P, P, P, P, P, P, i, i]
        L.oracle_precode.argtypes = [i, i, i, i, i, P, i, d, P, P, P, i, i]
        L.oracle_lmmse.argtypes = [i, i, i, i, i, i, d, P, P, P, P]
        L.oracle_zf.argtypes = [i, i, i, i, i, i, P, P, P]
        L.oracle_ml.argtypes = [i, i, i, P, P, i, P, P]
        L.oracle_learned_forward.argtypes = [i, i, i, i, i, P, i, d, i, P, P, P, P, P, P, P, i, i]
        L.oracle_learned_grad.argtypes = [i, i, i, i, i, P, i, d, i, P, P, P, P, P, P, P, i, i]
        for fn in (L.oracle_detect, L.oracle_precode, L.oracle_lmmse, L.oracle_zf, L.oracle_ml,
                   L.oracle_learned_forward, L.oracle_learned_grad):
            fn.restype = ctypes.c_int
        _lib = L
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _ranges(n, threads):
    threads = max(1, min(int(threads), n)) if n > 0 else 1
    step = (n + threads - 1) // threads if n > 0 else 0
    return [(s, min(n, s + step)) for s in range(0, n, step)] if n > 0 else [(0, 0)]


def _run(fn, n_sc, threads, call):
    rs = _ranges(n_sc, threads)
    if len(rs) == 1:
        rc = call(*rs[0])
        if rc != 0:
            raise RuntimeError(f"{fn} failed with status {rc}")
        return
    with _fut.ThreadPoolExecutor(len(rs)) as ex:
        for rc in ex.map(lambda r: call(*r), rs):
            if rc != 0:
                raise RuntimeError(f"{fn} failed with status {rc}")


def detect(H, Y, N0, cluster_size, K, Ex=1.0, fuse="colnorm", threads=1):
    """Algorithm 1 plus fusion.  Returns (Xhat [n_sc][n_sym][U], Xc [n_sc][C][n_sym][U], lam [n_sc][C])."""
    H = _c128(H)
    Y = _c128(Y)
    N0 = np.ascontiguousarray(N0, dtype=np.float64)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    cs = np.ascontiguousarray(cluster_size, dtype=np.int32)
    C = cs.size
    Xhat = np.zeros((n_sc, n_sym, U), np.complex128)
    Xc = np.zeros((n_sc, C, n_sym, U), np.complex128)
    lam = np.zeros((n_sc, C), np.float64)
    L = lib()
    _run("oracle_detect", n_sc, threads, lambda f0, f1: L.oracle_detect(
        n_sc, n_sym, B, U, C, _ptr(cs), int(K), float(Ex), FUSE[fuse], _ptr(H), _ptr(Y), _ptr(N0),
        _ptr(Xhat), _ptr(Xc), _ptr(lam), f0, f1))
    return Xhat, Xc, lam


def precode(H, S, cluster_size, K, rho=1.0, threads=1):
    """Algorithm 2 plus per-cluster power normalization.  Returns Xdl [n_sc][n_sym][B]."""
    H = _c128(H)
    S = _c128(S)
    n_sc, U, B = H.shape
    n_sym = S.shape[1]
    cs = np.ascontiguousarray(cluster_size, dtype=np.int32)
    Xdl = np.zeros((n_sc, n_sym, B), np.complex128)
    L = lib()
    _run("oracle_precode", n_sc, threads, lambda f0, f1: L.oracle_precode(
        n_sc, n_sym, B, U, cs.size, _ptr(cs), int(K), float(rho), _ptr(H), _ptr(S), _ptr(Xdl), f0, f1))
    return Xdl


def lmmse(H, Y, N0, Ex=1.0, rows=None):
    """Eq. (1) by Cholesky on antenna rows [r0, r0 + nr) (default: all, the centralized detector)."""
    H = _c128(H)
    Y = _c128(Y)
    N0 = np.ascontiguousarray(N0, dtype=np.float64)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    r0, nr = (0, B) if rows is None else rows
    X = np.zeros((n_sc, n_sym, U), np.complex128)
    rc = lib().oracle_lmmse(n_sc, n_sym, B, U, r0, nr, float(Ex), _ptr(H), _ptr(Y), _ptr(N0), _ptr(X))
    if rc != 0:
        raise RuntimeError(f"oracle_lmmse failed with status {rc}")
    return X


def zf(H, S, rows=None):
    """Local min-norm ZF, H^H (H H^H)^{-1} s, on antenna rows [r0, r0 + nr)."""
    H = _c128(H)
    S = _c128(S)
    n_sc, U, B = H.shape
    n_sym = S.shape[1]
    r0, nr = (0, B) if rows is None else rows
    X = np.zeros((n_sc, n_sym, nr), np.complex128)
    rc = lib().oracle_zf(n_sc, n_sym, B, U, r0, nr, _ptr(H), _ptr(S), _ptr(X))
    if rc != 0:
        raise RuntimeError(f"oracle_zf failed with status {rc}")
    return X


def ml(H, Y, points):
    """Exhaustive ML over points^U.  H: [n_vec][U][B], Y: [n_vec][B].  Returns labels [n_vec][U]."""
    H = _c128(H)
    Y = _c128(Y)
    pts = _c128(points)
    n_vec, U, B = H.shape
    lab = np.zeros((n_vec, U), np.int32)
    rc = lib().oracle_ml(n_vec, B, U, _ptr(H), _ptr(Y), pts.size, _ptr(pts), _ptr(lab))
    if rc != 0:
        raise RuntimeError(f"oracle_ml failed with status {rc}")
    return lab


def learned_param_count(K, U, hidden):
    """Length of the master parameter vector [tau(K), graw(K), W1(hidden*(U+1)), b1, w2, b2]."""
    return 2 * K + hidden * (U + 1) + 2 * hidden + 1


def learned_forward(H, Y, N0, cluster_size, K, master, hidden, Ex=1.0, threads=1):
    """Deep-unfolded CD with learned fusion.  Returns (Xhat, Xc, lam)."""
    H = _c128(H)
    Y = _c128(Y)
    N0 = np.ascontiguousarray(N0, dtype=np.float64)
    master = np.ascontiguousarray(master, dtype=np.float64)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    assert master.size == learned_param_count(K, U, hidden)
    cs = np.ascontiguousarray(cluster_size, dtype=np.int32)
    C = cs.size
    Xhat = np.zeros((n_sc, n_sym, U), np.complex128)
    Xc = np.zeros((n_sc, C, n_sym, U), np.complex128)
    lam = np.zeros((n_sc, C), np.float64)
    L = lib()
    _run("oracle_learned_forward", n_sc, threads, lambda f0, f1: L.oracle_learned_forward(
        n_sc, n_sym, B, U, C, _ptr(cs), int(K), float(Ex), int(hidden), _ptr(master), _ptr(H), _ptr(Y), _ptr(N0),
        _ptr(Xhat), _ptr(Xc), _ptr(lam), f0, f1))
    return Xhat, Xc, lam


def learned_grad(H, Y, N0, cluster_size, K, master, hidden, Xtarget, Ex=1.0):
    """Loss mean ||xhat - xtarget||^2 over vectors and its gradient w.r.t. the master parameters."""
    H = _c128(H)
    Y = _c128(Y)
    Xt = _c128(Xtarget)
    N0 = np.ascontiguousarray(N0, dtype=np.float64)
    master = np.ascontiguousarray(master, dtype=np.float64)
    n_sc, U, B = H.shape
    n_sym = Y.shape[1]
    cs = np.ascontiguousarray(cluster_size, dtype=np.int32)
    grad = np.zeros(master.size, np.float64)
    loss = np.zeros(1, np.float64)
    rc = lib().oracle_learned_grad(n_sc, n_sym, B, U, cs.size, _ptr(cs), int(K), float(Ex), int(hidden),
                                   _ptr(master), _ptr(H), _ptr(Y), _ptr(N0), _ptr(Xt), _ptr(loss), _ptr(grad), 0,
                                   n_sc)
    if rc != 0:
        raise RuntimeError(f"oracle_learned_grad failed with status {rc}")
    return float(loss[0]), grad
