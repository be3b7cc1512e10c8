"""Host-side model of the plane-pipeline 3D sweep's schedule (no GPU).

The kernel (csrc/sweep3dp.cuh) runs the warps of a CTA in lockstep chunks of
K = 4 steps with one barrier per chunk; warp (wy, h) runs 36 wy + 4 h steps
behind warp (0, 0).  Values cross warps through shared-memory rings (z: depth
8 virtual columns, all lanes; y: depth 16, lane 31 -> lane 0) and, between
passes of H planes, through a global buffer that the first warp of a pass
reads two steps ahead.  These tests replay that schedule step by step and
check, for every value a cell of the grid reads from another warp, that it
was written in an earlier chunk by the right producer and not overwritten
before the read; they also check that the skewed per-cell layout is a
bijection whose 32 cells of a warp step are consecutive, and that the
partial-sum tile, written 4 rows per chunk, stores every cell exactly once.
The constants below restate the kernel's.
"""
import math

import pytest

K, RZ, RY = 4, 8, 16
LY, LZ = 32 + K, K


def heights(nx, ny, nz):
    wy = -(-ny // 32)
    return [H for H in range(1, 17)
            if wy * H <= 16 and H <= nz and not (-(-nz // H) > 1 and (H < 2 or nx < 4 * H + 2))]


def hazards(nx, ny, nz, H, prefetch=2):
    """Number of reads that would see a wrong or racing value."""
    WY = -(-ny // 32)
    M = -(-nz // H)
    U = M * nx
    n_loc = (U + 62) & ~31
    writes = {"z": {}, "y": {}, "w": {}}
    reads = []
    for wy in range(WY):
        for h in range(H):
            d = wy * LY + h * LZ
            for tau in range(n_loc):
                g = d + tau
                for lam in range(32):
                    u = tau - lam
                    j = 32 * wy + lam
                    inside = 0 <= u < U
                    m, i = divmod(u, nx) if inside else (None, None)
                    cell = inside and j < ny and h + H * m < nz
                    if h < H - 1:
                        writes["z"].setdefault((wy, h, u % RZ, lam), []).append((g, u))
                    if h > 0 and cell:
                        reads.append(("z", (wy, h - 1, u % RZ, lam), g, u))
                    if lam == 31 and wy < WY - 1:
                        writes["y"].setdefault((wy, h, u % RY), []).append((g, u))
                    if lam == 0 and wy > 0 and cell:
                        reads.append(("y", (wy - 1, h, u % RY), g, u))
                    if M > 1 and h == H - 1 and cell and m + 1 < M:
                        writes["w"].setdefault((i, j), []).append((g, (m, i, j)))
                    if M > 1 and h == 0 and cell and m >= 1:
                        reads.append(("w", (i, j), g - prefetch, (m - 1, i, j)))
    bad = 0
    for kind, key, g, expect in reads:
        chunk = g // K
        ws = writes[kind].get(key, [])
        before = [x for x in ws if x[0] // K < chunk]
        same = [x for x in ws if x[0] // K == chunk]
        if not before or max(before)[1] != expect or same:
            bad += 1
    return bad


SHAPES = [(4, 3, 3), (6, 5, 4), (22, 40, 19), (26, 35, 23), (40, 9, 2), (10, 33, 7), (18, 70, 11)]


@pytest.mark.parametrize("n", SHAPES, ids=["x".join(map(str, s)) for s in SHAPES])
def test_no_hazards_for_every_accepted_height(n):
    for H in heights(*n):
        assert hazards(*n, H) == 0, H


def test_model_detects_a_too_short_row():
    """nx < 4 H + 2 (refused by the runtime) does break the wrap link."""
    assert hazards(9, 33, 7, 2) > 0
    assert hazards(12, 40, 9, 3, prefetch=5) > 0


def skew_index(nx, ny, nz, f, X, Y, Z):
    """Rows along y: row coordinate Y, plane coordinate Z (for rows along z
    call it with the roles of y and z exchanged)."""
    nyp = 32 * (-(-ny // 32))
    nd = nx + ny - 1
    fam = nz * nd * nyp
    key = X + (ny - 1 - Y) if f else X + Y
    return f * fam + (Z * nd + key) * nyp + Y


@pytest.mark.parametrize("n", [(22, 40, 19), (26, 35, 23), (16, 80, 6)])
def test_skewed_layout(n):
    nx, ny, nz = n
    nyp = 32 * (-(-ny // 32))
    fam = nz * (nx + ny - 1) * nyp
    for f in (0, 1):
        idx = {skew_index(nx, ny, nz, f, X, Y, Z) for Z in range(nz) for Y in range(ny) for X in range(nx)}
        assert len(idx) == nx * ny * nz and min(idx) >= f * fam and max(idx) < (f + 1) * fam
    # the cells of one warp step (one pass) are consecutive entries, for every octant
    H = heights(*n)[-1]
    M = -(-nz // H)
    for neg in range(8):
        negx, negy, negz = neg & 1, (neg >> 1) & 1, (neg >> 2) & 1
        f = 1 if negx != negy else 0
        for wy in range(-(-ny // 32)):
            for h in range(H):
                for tau in range(0, M * nx + 31, 5):
                    by_pass = {}
                    for lam in range(32):
                        u, j = tau - lam, 32 * wy + lam
                        if u < 0 or u >= M * nx or j >= ny:
                            continue
                        m, i = divmod(u, nx)
                        k = h + H * m
                        if k >= nz:
                            continue
                        X = nx - 1 - i if negx else i
                        Y = ny - 1 - j if negy else j
                        Z = nz - 1 - k if negz else k
                        by_pass.setdefault(m, []).append(skew_index(nx, ny, nz, f, X, Y, Z))
                    for offs in by_pass.values():
                        assert max(offs) - min(offs) == len(offs) - 1


@pytest.mark.parametrize("n,H", [((22, 40, 19), 5), ((64, 64, 64), 4), ((10, 33, 7), 2)])
def test_tile_rows_written_once(n, H):
    nx, ny, nz = n
    WY = -(-ny // 32)
    M = -(-nz // H)
    U = M * nx
    n_loc = (U + 62) & ~31
    for wy in range(WY):
        for h in range(H):
            seen = {}
            for tau0 in range(0, n_loc, K):
                te = tau0 + K - 1
                g = (te >> 2) & 7
                for lane in range(32):
                    tq = te - ((te - lane) & 31)
                    u_top = tq - 4 * g
                    m = math.floor((u_top + 0.5) / nx)
                    i = u_top - m * nx
                    for q in range(4):
                        if q:
                            i -= 1
                            if i < 0:
                                i += nx
                                m -= 1
                        if m >= 0 and h + H * m < nz and 32 * wy + 4 * g + q < ny:
                            key = (4 * g + q, m * nx + i)
                            assert m * nx + i == tq - (4 * g + q)
                            seen[key] = seen.get(key, 0) + 1
            for r in range(32):
                if 32 * wy + r >= ny:
                    continue
                for u in range(U):
                    if h + H * (u // nx) < nz:
                        assert seen.get((r, u)) == 1
