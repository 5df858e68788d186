"""Shared-memory layout rules of the tensor-core kernel, checked on the host: with the row padding
(c64 rows of 2 B_c + 8 words, 16-bit rows of B_c + 4 words) and the tile-row stride (>= n_tiles,
4 mod 16 entries), the fragment loads the MMAs issue fall on distinct banks, as the kernel's layout
comment states.

A warp's lane l is (gid, tig) = (l // 4, l % 4).  32-bit accesses are served per warp (32 banks of
4 bytes); 64-bit accesses per half-warp (16 lanes), an 8-byte word covering two banks.  Lanes that
read the same address share it (broadcast).
"""
import os

PLAN_H = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1902_08653_gb300",
                           "csrc", "plan.h")).read()


def test_rules_are_the_library_ones():
    """The two formulas below restate plan.h's."""
    assert "return ((unsigned)n_tiles + 11u) / 16u * 16u + 4u;" in PLAN_H
    assert "return in_dtype == CDMIMO_C64 ? 2u * (unsigned)Bc + 8u : (unsigned)Bc + 4u;" in PLAN_H


def row_words(Bc, c64):
    """Words per channel row (plan.h: tc_row_words)."""
    return 2 * Bc + 8 if c64 else Bc + 4


def tile_stride(n_tiles):
    """Tile-row stride in complex entries (plan.h: tc_x_stride)."""
    return (n_tiles + 11) // 16 * 16 + 4


def conflict_degree_64(addr8):
    """Worst bank conflict of a warp's 64-bit accesses, addr8[lane] in 8-byte units."""
    worst = 1
    for half in (range(0, 16), range(16, 32)):
        by_bank = {}
        for l in half:
            by_bank.setdefault(addr8[l] % 16, set()).add(addr8[l])
        worst = max(worst, max(len(v) for v in by_bank.values()))
    return worst


def conflict_degree_32(addr4):
    by_bank = {}
    for l in range(32):
        by_bank.setdefault(addr4[l] % 32, set()).add(addr4[l])
    return max(len(v) for v in by_bank.values())


LANES = [(l // 4, l % 4) for l in range(32)]


def test_row_and_stride_rules():
    for Bc in (16, 32):
        assert row_words(Bc, True) % 32 == 8  # 8-byte entries: row stride 4 mod 16 entries
        assert (row_words(Bc, True) * 4) % 16 == 0 and (row_words(Bc, False) * 4) % 16 == 0  # bulk-copy rows
    for n_tiles in range(1, 300):
        xs = tile_stride(n_tiles)
        assert xs >= n_tiles and xs % 16 == 4


def test_c64_fragment_loads_are_conflict_free():
    for Bc in (16, 32):
        sr2 = row_words(Bc, True) // 2  # row stride in complex (8-byte) entries
        for ks in range(Bc // 4):
            # phase A: A fragment rows gid / gid + 8 and Gram B fragment rows 8 j + gid, entry 4 ks + tig
            for r0 in (0, 8):
                assert conflict_degree_64([(gid + r0) * sr2 + 4 * ks + tig for gid, tig in LANES]) == 1
        for ks in range(4):
            # phase C: H^T fragment, user 4 ks + tig, antennas 16 m + gid (+8)
            for m in range(Bc // 16):
                for off in (0, 8):
                    a = [(4 * ks + tig) * sr2 + 16 * m + gid + off for gid, tig in LANES]
                    assert conflict_degree_64(a) == 1


def test_tile_rows_w_loads_are_conflict_free():
    for n_sym, C in ((14, 8), (16, 8), (8, 16), (5, 6)):
        xs = tile_stride(C * n_sym)
        for c in range(C):
            for ks in range(4):
                for j in range(2):
                    a = [(4 * ks + tig) * xs + c * n_sym + 8 * j + gid for gid, tig in LANES]
                    assert conflict_degree_64(a) == 1


def test_16bit_rows():
    for Bc in (16, 32):
        sw = row_words(Bc, False)  # one word per complex entry
        for ks in range(Bc // 4):
            for r0 in (0, 8):  # phase A: conflict-free
                assert conflict_degree_32([(gid + r0) * sw + 4 * ks + tig for gid, tig in LANES]) == 1
        for ks in range(4):  # phase C: at most two-way, as the plan's comment says
            for m in range(Bc // 16):
                a = [(4 * ks + tig) * sw + 16 * m + gid for gid, tig in LANES]
                assert conflict_degree_32(a) <= 2
