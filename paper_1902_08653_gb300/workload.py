"""Seeded synthetic workloads for decentralized CD detection and precoding.

This module is shared by the CUDA path's tests and benchmarks and by the FP64 oracle's tests.  It
holds no arithmetic of the detection / precoding method itself: only the system model that produces
the inputs (Sec. II: i.i.d. Rayleigh channel, QAM symbols, AWGN, y = H x + n), the constellation
labelling used to count bit errors, and the 16-bit storage format of the reduced-precision inputs.

Array layouts (row-major, complex = interleaved re/im):
  H  [n_sc][U][B]      uplink channel; row u holds column h_u of H^ul (the paper's B x U matrix),
                       so h_{u,c} = H[f, u, o_c:o_c+B_c] is contiguous.  H^dl = (H^ul)^H (Sec. II-B).
  X  [n_sc][n_sym][U]  transmitted uplink symbols (Ex = 1).
  Y  [n_sc][n_sym][B]  received uplink vectors, y = H^ul x + n  (Sec. II-A).
  S  [n_sc][n_sym][U]  downlink symbol vectors s.
  N0 [n_sc]            noise variance per receive antenna.

Seeds: every draw comes from numpy's Philox bit generator keyed by (seed, tag), so a workload is a
pure function of its arguments.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20190222


def rng(seed: int, tag: int = 0) -> np.random.Generator:
    """Counter-based generator keyed by (seed, tag)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(tag)])))


# --------------------------------------------------------------------------------------------
# constellations (the paper uses 16-QAM, Sec. V; Gray labelling is our reading: it is silent)
# --------------------------------------------------------------------------------------------
def _gray(i):
    return i ^ (i >> 1)


def qam(M: int):
    """Gray-labelled square M-QAM with unit average energy (Ex = 1).

    Returns (points[M] complex128, L, scale): points[label], L levels per axis, and the factor that
    maps the integer grid {-(L-1), ..., L-1} onto the unit-energy constellation.  A label's high
    log2(L) bits select the in-phase level and its low bits the quadrature level, each Gray-coded.
    """
    L = int(round(np.sqrt(M)))
    if L * L != M or L < 2 or (L & (L - 1)):
        raise ValueError(f"M={M} is not a square power-of-4 QAM order")
    k = L.bit_length() - 1
    inv = np.empty(L, dtype=np.int64)
    for i in range(L):
        inv[_gray(i)] = i
    scale = 1.0 / np.sqrt(2.0 * (L * L - 1) / 3.0)
    labels = np.arange(M)
    li = inv[labels >> k]
    lq = inv[labels & (L - 1)]
    pts = ((2 * li - (L - 1)) + 1j * (2 * lq - (L - 1))) * scale
    return pts.astype(np.complex128), L, scale


def hard_decision(x: np.ndarray, M: int):
    """Nearest-point slicing of raw estimates (no de-biasing; an unstated detail, our reading).

    Returns (labels, margin): margin is the per-entry distance to the closest decision threshold
    over both axes, in the same units as x, so that decisions whose margin is tiny can be excluded
    from an exact-match comparison.
    """
    _, L, scale = qam(M)
    k = L.bit_length() - 1
    out = []
    margins = []
    for comp in (np.real(x), np.imag(x)):
        v = np.asarray(comp, dtype=np.float64) / scale
        lev = np.clip(np.round((v + (L - 1)) / 2.0), 0, L - 1).astype(np.int64)
        thr = np.arange(L - 1) * 2.0 - (L - 2)  # midpoints between adjacent levels
        d = np.min(np.abs(v[..., None] - thr), axis=-1) * scale
        out.append(_gray(lev))
        margins.append(d)
    labels = (out[0] << k) | out[1]
    return labels, np.minimum(margins[0], margins[1])


def bit_errors(labels_a: np.ndarray, labels_b: np.ndarray) -> int:
    """Number of differing label bits between two label arrays."""
    diff = np.ascontiguousarray(np.bitwise_xor(np.asarray(labels_a, dtype=np.uint64),
                                               np.asarray(labels_b, dtype=np.uint64)))
    return int(np.unpackbits(diff.view(np.uint8)).sum())


# --------------------------------------------------------------------------------------------
# system model
# --------------------------------------------------------------------------------------------
def snr_to_n0(snr_db, U: int, Ex: float = 1.0):
    """Per-receive-antenna SNR = E||H x||^2 / E||n||^2 = U Ex / N0 (our reading; paper silent)."""
    return U * Ex * 10.0 ** (-np.asarray(snr_db, dtype=np.float64) / 10.0)


def rayleigh(g: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. CN(0, 1) entries (Sec. V: Rayleigh fading)."""
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return ((re + 1j * im) * np.sqrt(0.5)).astype(np.complex128)


def symbols(g: np.random.Generator, M: int, shape):
    pts, _, _ = qam(M)
    lab = g.integers(0, M, size=shape)
    return pts[lab], lab


def uplink(seed: int, n_sc: int, n_sym: int, B: int, U: int, snr_db=10.0, M: int = 16, tag: int = 1):
    """Uplink batch: H fixed over the n_sym symbols of a subcarrier, fresh x and n per symbol.

    snr_db may be a scalar or an array of per-subcarrier SNRs.  Returns a dict of complex128 /
    float64 numpy arrays (H, X, labels, Y, N0).
    """
    g = rng(seed, tag)
    H = rayleigh(g, (n_sc, U, B))
    X, lab = symbols(g, M, (n_sc, n_sym, U))
    snr = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (n_sc,))
    N0 = snr_to_n0(snr, U)
    noise = rayleigh(g, (n_sc, n_sym, B)) * np.sqrt(N0)[:, None, None]
    Y = np.einsum("fub,fnu->fnb", H, X) + noise
    return {"H": H, "X": X, "labels": lab, "Y": Y, "N0": N0, "snr_db": snr.copy(), "M": M}


def downlink(seed: int, n_sc: int, n_sym: int, B: int, U: int, M: int = 16, tag: int = 2):
    """Downlink batch: channel H (uplink layout; H^dl = H^H by reciprocity) and symbols s."""
    g = rng(seed, tag)
    H = rayleigh(g, (n_sc, U, B))
    S, lab = symbols(g, M, (n_sc, n_sym, U))
    return {"H": H, "S": S, "labels": lab, "M": M}


def sweep_snr(n_sc: int, snrs=(0, 5, 10, 15, 20, 25, 30)):
    """Per-subcarrier SNR that cycles through an SNR sweep, so one batch covers every point."""
    s = np.asarray(snrs, dtype=np.float64)
    return s[np.arange(n_sc) % len(s)]


def partition(B: int, C: int):
    """Uniform partition of B antennas into C contiguous clusters (B_c = B / C, Sec. II-A)."""
    if B % C:
        raise ValueError("B must be divisible by C for a uniform partition")
    return [B // C] * C


# --------------------------------------------------------------------------------------------
# 16-bit storage with a per-subcarrier FP32 scale (reduced-precision inputs)
# --------------------------------------------------------------------------------------------
def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP32 -> bfloat16 bit pattern (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rnd = ((u >> 16) & 1) + 0x7FFF
    return ((u + rnd) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def quantize_c16(A: np.ndarray, kind: str):
    """Store complex A [n_sc, ...] as 16-bit complex (kind 'f16' or 'bf16') with scale a_f.

    a_f = sqrt(mean |A_f|^2) over each subcarrier's entries; the stored value is A_f / a_f.  Returns
    (q, scale, deq): q is an [..., 2] uint16 array (bit patterns, re/im interleaved), scale is
    float32 [n_sc], and deq = scale * float(q) is the exact complex128 value the stored data encodes,
    which is what both the CUDA path and the oracle must be given to be compared.
    """
    n_sc = A.shape[0]
    flat = A.reshape(n_sc, -1)
    scale = np.sqrt(np.mean(np.abs(flat) ** 2, axis=1)).astype(np.float32)
    scale = np.where(scale > 0, scale, np.float32(1.0)).astype(np.float32)
    norm = (A / scale.reshape((n_sc,) + (1,) * (A.ndim - 1)).astype(np.float64))
    pair = np.stack([norm.real, norm.imag], axis=-1).astype(np.float32)
    if kind == "f16":
        q = pair.astype(np.float16).view(np.uint16)
        back = q.view(np.float16).astype(np.float64)
    elif kind == "bf16":
        q = f32_to_bf16_bits(pair)
        back = bf16_bits_to_f32(q).astype(np.float64)
    else:
        raise ValueError(kind)
    deq = (back[..., 0] + 1j * back[..., 1]) * scale.reshape((n_sc,) + (1,) * (A.ndim - 1)).astype(np.float64)
    return q, scale, deq


def as_c64(A: np.ndarray) -> np.ndarray:
    """complex64 copy of A, and (as second value) the complex128 value the complex64 data holds."""
    a32 = np.ascontiguousarray(A, dtype=np.complex64)
    return a32, a32.astype(np.complex128)


# --------------------------------------------------------------------------------------------
# uneven resource blocks (batched launches)
# --------------------------------------------------------------------------------------------
def random_partition(g: np.random.Generator, B: int, sizes=(16, 32, 64)):
    """A seeded random sequence of cluster sizes from `sizes` that sums to B."""
    cs, rem = [], B
    while rem > 0:
        opts = [s for s in sizes if s <= rem]
        if not opts:
            raise ValueError("B cannot be partitioned into the given sizes")
        s = int(g.choice(opts))
        cs.append(s)
        rem -= s
    return cs


def resource_blocks(seed: int, n_rb: int = 100, n_sc: int = 12, n_sym: int = 14, Bs=(128, 256, 512),
                    sizes=(16, 32, 64), U_range=(8, 64), snr_db=20.0, M: int = 16, downlink_too: bool = False):
    """Uneven resource blocks: per block B uniform from Bs, a random partition into `sizes`, U uniform
    in U_range (inclusive), n_sc subcarriers x n_sym symbols of uplink data (and downlink symbols if
    asked).  Returns a list of dicts: B, U, cluster_size and the uplink (and downlink) arrays."""
    g = rng(seed, 4)
    out = []
    for r in range(n_rb):
        B = int(g.choice(Bs))
        cs = random_partition(g, B, sizes)
        U = int(g.integers(U_range[0], U_range[1] + 1))
        blk = {"B": B, "U": U, "cluster_size": cs}
        blk.update(uplink(seed * 100003 + r, n_sc, n_sym, B, U, snr_db=snr_db, M=M, tag=5))
        if downlink_too:
            dl = downlink(seed * 100003 + r, n_sc, n_sym, B, U, M=M, tag=6)
            blk["S"] = dl["S"]
        out.append(blk)
    return out


# --------------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): the host twin of the device generator
# --------------------------------------------------------------------------------------------
_PHILOX_M = (np.uint64(0xD2511F53), np.uint64(0xCD9E8D57))
_PHILOX_W = (np.uint32(0x9E3779B9), np.uint32(0xBB67AE85))


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorized Philox4x32-10 on uint32 arrays (counter words c0..c3, key words k0, k1)."""
    c = [np.asarray(v, dtype=np.uint32).copy() for v in (c0, c1, c2, c3)]
    k = [np.asarray(k0, dtype=np.uint32).copy(), np.asarray(k1, dtype=np.uint32).copy()]
    m32 = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k[0] = (k[0].astype(np.uint64) + np.uint64(_PHILOX_W[0])).astype(np.uint32)
            k[1] = (k[1].astype(np.uint64) + np.uint64(_PHILOX_W[1])).astype(np.uint32)
        p0 = _PHILOX_M[0] * c[0].astype(np.uint64)
        p1 = _PHILOX_M[1] * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & m32).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & m32).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return c


def philox_stream(seed: int, stream: int, n: int):
    """The four output words for elements 0..n-1 of a stream (counter (lo(i), hi(i), stream, 0))."""
    i = np.arange(n, dtype=np.uint64)
    return philox4x32_10((i & np.uint64(0xFFFFFFFF)).astype(np.uint32), (i >> np.uint64(32)).astype(np.uint32),
                         np.full(n, stream, np.uint32), np.zeros(n, np.uint32),
                         np.full(n, seed & 0xFFFFFFFF, np.uint32), np.full(n, (seed >> 32) & 0xFFFFFFFF, np.uint32))


def philox_cnormal(seed: int, stream: int, n: int, var=1.0):
    """CN(0, var) samples by Box-Muller from the first two words, u = (w + 0.5) / 2^32 (FP64)."""
    w = philox_stream(seed, stream, n)
    u1 = (w[0].astype(np.float64) + 0.5) / 2.0 ** 32
    u2 = (w[1].astype(np.float64) + 0.5) / 2.0 ** 32
    rad = np.sqrt(-2.0 * np.log(u1) * 0.5 * np.asarray(var, dtype=np.float64))
    return rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)


def philox_uplink(seed: int, n_sc: int, n_sym: int, B: int, U: int, snr_db, M: int = 16):
    """The batch cdmimo_synth_uplink draws, computed on the host in FP64 (for tests)."""
    H = philox_cnormal(seed, 0, n_sc * U * B).reshape(n_sc, U, B)
    lab = (philox_stream(seed, 1, n_sc * n_sym * U)[0] & np.uint32(M - 1)).astype(np.int64).reshape(n_sc, n_sym, U)
    pts, _, _ = qam(M)
    X = pts[lab]
    N0 = snr_to_n0(np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (n_sc,)), U)
    noise = philox_cnormal(seed, 2, n_sc * n_sym * B, var=np.repeat(N0, n_sym * B)).reshape(n_sc, n_sym, B)
    Y = np.einsum("fub,fnu->fnb", H, X) + noise
    return {"H": H, "X": X, "labels": lab, "Y": Y, "N0": N0, "noise": noise}
