"""Shared-memory positions of the z-marching passes (no GPU).

The position formulas of cg27_step.cuh, restated: every tile shape in use gets
its tile-plus-halo array covered exactly once, with slot 0 of every thread its
own tile cell where the pass relies on it, and every stencil read window of a
tile cell inside the array -- so no shared-memory access of these passes
leaves its array, whatever the launch shape.
"""
import pytest

SHAPES = [(32, 8), (32, 4), (32, 16)]


def ring_slots(tx_n, ty_n, h):
    """RingSlots<H, Shape<TX, TY>>: (thread, slot) -> (lx, ly)."""
    W = tx_n + 2 * h
    PL = W * (ty_n + 2 * h)
    NT = tx_n * ty_n
    NR = PL - NT
    K = 1 + (NR + NT - 1) // NT
    pos = {}
    for tid in range(NT):
        tx, ty = tid % tx_n, tid // tx_n
        for k in range(K):
            if k == 0:
                lx, ly = tx + h, ty + h
            else:
                r = tid + (k - 1) * NT
                if r < h * W:
                    lx, ly = r % W, r // W
                elif r < 2 * h * W:
                    lx, ly = (r - h * W) % W, ty_n + h + (r - h * W) // W
                elif r < NR:
                    q = r - 2 * h * W
                    row, col = q // (2 * h), q % (2 * h)
                    lx = col if col < h else tx_n + col
                    ly = h + row
                else:
                    continue
            pos[(tid, k)] = (lx, ly)
    return pos, W, ty_n + 2 * h


def halo_slots(tx_n, ty_n, h, nt=None):
    """HaloSlots<HALO, Shape<TX, TY>, NTB>: position i = tid + k NTB of the array."""
    W = tx_n + 2 * h
    PL = W * (ty_n + 2 * h)
    NT = nt or tx_n * ty_n
    K = (PL + NT - 1) // NT
    return {(tid, k): ((tid + k * NT) % W, (tid + k * NT) // W)
            for tid in range(NT) for k in range(K) if tid + k * NT < PL}, W, ty_n + 2 * h


def _covers_once(pos, W, H):
    seen = sorted(pos.values())
    assert seen == sorted((x, y) for x in range(W) for y in range(H))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("h", [1, 2])
def test_ring_slots_cover_the_array_once_with_the_own_cell_first(shape, h):
    tx_n, ty_n = shape
    pos, W, H = ring_slots(tx_n, ty_n, h)
    _covers_once(pos, W, H)
    for tid in range(tx_n * ty_n):
        assert pos[(tid, 0)] == (tid % tx_n + h, tid // tx_n + h)


@pytest.mark.parametrize("shape", SHAPES)
def test_halo_slots_cover_the_array_once(shape):
    pos, W, H = halo_slots(*shape, 1)
    _covers_once(pos, W, H)


def test_divergence_blocks_of_352_threads():
    """k_div_sep runs 352 threads on a 32 x 8 tile: one slot per thread covers
    the 340 positions of tile plus halo once, and the threads that form an
    output cell (rows below 8) are exactly the tile's 256."""
    pos, W, H = halo_slots(32, 8, 1, nt=352)
    _covers_once(pos, W, H)
    assert max(k for _, k in pos) == 0
    out = [tid for tid in range(352) if tid // 32 < 8]
    assert len(out) == 256 and all((tid % 32 + 1, tid // 32 + 1) in set(pos.values()) for tid in out)


@pytest.mark.parametrize("shape", SHAPES)
def test_stencil_windows_stay_inside(shape):
    """The field pass reads 3 x 3 windows of the phi pairs around every n
    position (halo 1 inside halo 2) and of the n records around every tile
    cell; the divergence and macroscopic passes read 3 x 3 windows around
    every tile cell of their halo-1 arrays."""
    tx_n, ty_n = shape
    pos1, W1, H1 = ring_slots(tx_n, ty_n, 1)
    _, W2, H2 = ring_slots(tx_n, ty_n, 2)
    for (lx, ly) in pos1.values():  # n position -> phi-pair window (shifted by one)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                x, y = lx + 1 + dx, ly + 1 + dy
                assert 0 <= x < W2 and 0 <= y < H2
    for tid in range(tx_n * ty_n):
        cx, cy = tid % tx_n + 1, tid // tx_n + 1
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                assert 0 <= cx + dx < W1 and 0 <= cy + dy < H1


def test_fused_pass_positions():
    """k_collide_macro: 340 positions of a 32 x 8 tile with its ring, tile
    cells first (tid < 256), then the top row, the bottom row and both ends of
    the rows between; the 27 gathered sources of every tile cell lie inside."""
    FX, FY = 32, 8
    FW, FH = FX + 2, FY + 2
    FPL = FW * FH
    FNT = (FPL + 31) // 32 * 32
    assert FNT == 352
    pos = []
    for tid in range(FPL):
        if tid < FX * FY:
            lx, ly = tid % FX + 1, tid // FX + 1
        else:
            r = tid - FX * FY
            if r < FW:
                lx, ly = r, 0
            elif r < 2 * FW:
                lx, ly = r - FW, FH - 1
            else:
                lx, ly = (FW - 1 if (r - 2 * FW) & 1 else 0), 1 + (r - 2 * FW) // 2
        pos.append((lx, ly))
    assert sorted(pos) == sorted((x, y) for x in range(FW) for y in range(FH))
    for tid in range(FX * FY):
        lx, ly = pos[tid]
        p = lx + FW * ly
        for cx in (-1, 0, 1):
            for cy in (-1, 0, 1):
                assert 0 <= p - cx - FW * cy < FPL
