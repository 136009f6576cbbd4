"""Shared-memory bank model of the region kernel's evolution (CPU only).

The kernel takes the cells of a level in 2x2x2 blocks (block index z fastest,
then x, then y; eight consecutive threads per block) and keeps (pi, c) in
slots whose x bits 1-2 are flipped by the y and z parities (pc_slot).  These
tests replay that order for every level of every region type from the
planner's active boxes and count shared-memory wavefronts per warp access
(32 banks of 4 bytes; a wavefront serves at most one distinct word per bank),
against the ideal (bytes / 128 per access).  They pin the property the layout
was chosen for: the seven phi reads, the phi write and the (pi, c) read and
write of a warp cost close to the minimum, where the plain row-major order cost
about 1.5x.
"""
import ctypes

import numpy as np
import pytest


def _wavefronts(words):
    """words: int array [lanes, k] of 4-byte word addresses of one warp access."""
    w = np.unique(words.ravel())
    return int(np.bincount(w % 32, minlength=32).max())


def _pc_slot(x, y, z, B):
    return (z * B + y) * B + (x ^ ((((y & 1) << 1) | ((z & 1) << 2)) & (B - 1)))


def _level_cells(lo, hi, order):
    w0, w1, w2 = (hi[d] - lo[d] for d in range(3))
    n = w0 * w1 * w2
    j = np.arange(n)
    if order == "block":
        a, c = w0 // 2, w2 // 2
        m, corner = j >> 3, j & 7
        r = m // c
        jj = r // a
        ux = lo[0] + 2 * (r - jj * a) + (corner & 1)
        uy = lo[1] + 2 * jj + ((corner >> 1) & 1)
        uz = lo[2] + 2 * (m - r * c) + ((corner >> 2) & 1)
    else:  # row-major, x fastest
        ux = lo[0] + j % w0
        uy = lo[1] + (j // w0) % w1
        uz = lo[2] + j // (w0 * w1)
    return ux, uy, uz


def _count(rx, B, order, swizzle):
    P = B + 2
    got = ideal = 0
    cells_seen = 0
    lohi = (ctypes.c_int32 * 6)()
    for S in range(8):
        levels = rx.rx_active_box(B, S, 0, lohi)
        assert levels > 0
        for k in range(1, levels + 1):
            rx.rx_active_box(B, S, k, lohi)
            lo, hi = list(lohi[:3]), list(lohi[3:])
            if min(h - l for l, h in zip(lo, hi)) <= 0:
                continue
            ux, uy, uz = _level_cells(lo, hi, order)
            cells_seen += len(ux)
            pidx = (uz * P + uy) * P + ux
            x, y, z = ux - 1, uy - 1, uz - 1
            cidx = _pc_slot(x, y, z, B) if swizzle else (z * B + y) * B + x
            for w in range(0, len(pidx), 32):
                p, c = pidx[w:w + 32], cidx[w:w + 32]
                n = len(p)
                for off in (0, -1, 1, -P, P, -P * P, P * P, 0):  # 7 reads + the write
                    got += _wavefronts(np.stack([2 * (p + off), 2 * (p + off) + 1], 1))
                    ideal += -(-n * 8 // 128)
                for _ in range(2):  # (pi, c) read and write
                    got += _wavefronts(np.stack([4 * c + i for i in range(4)], 1))
                    ideal += -(-n * 16 // 128)
    return got, ideal, cells_seen


@pytest.mark.parametrize("B", [8, 16])
def test_block_order_is_near_conflict_free(rx, B):
    got, ideal, cells = _count(rx, B, "block", True)
    assert cells == (B // 2) * B ** 3  # every cell of a period cell, every level
    assert got <= 1.10 * ideal, (got, ideal)


def test_row_major_order_was_not(rx):
    """The order the block layout replaced: its conflicts are what it removes."""
    got_row, ideal, _ = _count(rx, 16, "row", False)
    got_blk, _, _ = _count(rx, 16, "block", True)
    assert got_row >= 1.4 * ideal
    assert got_blk < 0.8 * got_row


def test_block_without_slot_swizzle_conflicts_on_pi_c(rx):
    """Without the swizzle the eight (pi, c) slots of a block fall into two
    16-byte bank groups."""
    got_plain, ideal, _ = _count(rx, 16, "block", False)
    got_swz, _, _ = _count(rx, 16, "block", True)
    assert got_plain > 1.3 * got_swz
