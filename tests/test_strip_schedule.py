"""The row-strip two-step kernel's schedule, replayed on the CPU: its ring-slot formula, the
gather and push columns (rows of any width: a block's pairs cover the row rounded up to 64
columns, a row of odd width ends on a lone node whose partner is read from the padding and
dropped), the split of the running rows into one range per block, and the partial-sum slots the
last block adds.  The kernel's index arithmetic is mirrored here (the
CUDA source is not imported); every access is checked against its buffer, each destination of
the push must be written exactly once, and one launch must equal two plain collide-and-stream
steps, also when a thread runs one row ahead and writes the next phase-A row before a slower
thread gathers (the case the slot counts 4 / 3 / 2 of the c_y = +1 / 0 / -1 groups are for)."""
import numpy as np
import pytest

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
PLANES = 27


def collide(g, omega):
    """BGK on shifted populations g = f - w, [9, n], FP64."""
    drho = g.sum(0)
    jx = sum(CX[i] * g[i] for i in range(9))
    jy = sum(CY[i] * g[i] for i in range(9))
    rho = 1.0 + drho
    ux, uy = jx / rho, jy / rho
    out = np.empty_like(g)
    for i in range(9):
        cu = CX[i] * ux + CY[i] * uy
        geq = W[i] * (drho + rho * (3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)))
        out[i] = g[i] + omega * (geq - g[i])
    return out


def two_plain_steps(f, omega):
    for _ in range(2):
        c = collide(f.reshape(9, -1), omega).reshape(f.shape)
        f = np.stack([np.roll(np.roll(c[i], CY[i], 0), CX[i], 1) for i in range(9)])
    return f


def strip_plane(i, q):
    """Ring plane of direction i for the phase-A row with sequence number q."""
    group, k = {2: (0, 0), 5: (0, 1), 6: (0, 2), 0: (1, 0), 1: (1, 1), 3: (1, 2), 4: (2, 0), 7: (2, 1),
                8: (2, 2)}[i]
    if group == 0:
        return (q & 3) * 3 + k
    if group == 1:
        return 12 + (q % 3) * 3 + k
    return 21 + (q & 1) * 3 + k


def launch(nx, nys, grid, race, seed):
    rng = np.random.default_rng(seed)
    omega = 1.3
    row_base = np.concatenate([[0], np.cumsum(nys)]).astype(int)
    rows = int(row_base[-1])
    # rows padded to whole 64-column blocks; the padding holds NaN, so a value read from it (the
    # dropped partner of a lone node) shows in any result it reaches
    np_ = ((nx + 1) // 2 + 31) // 32 * 32  # threads: one per node pair, whole warps
    rw = 2 * np_                            # ring width (and padded row)
    src = []
    for ny in nys:
        a = np.full((9, ny, rw), np.nan)
        a[:, :, :nx] = rng.normal(0.0, 0.01, (9, ny, nx))
        src.append(a)
    dst = [np.full((9, ny, nx), np.nan) for ny in nys]
    writes = [np.zeros((9, ny, nx), int) for ny in nys]
    per = (rows + grid - 1) // grid
    starts = set()
    x = 2 * np.arange(np_)
    va, vb = x < nx, x + 1 < nx
    xl = np.where(x == 0, nx - 1, x - 1)
    xar = np.where(x + 1 >= nx, x + 1 - nx, x + 1)
    xbr = np.where(x + 2 >= nx, x + 2 - nx, x + 2)
    for b in range(grid):
        r0, r1 = b * per, min(rows, b * per + per)
        r = r0
        while r < r1:
            j = max(k for k in range(len(nys)) if row_base[k] <= r)
            rb, ny = int(row_base[j]), nys[j]
            ya, yb = r - rb, min(ny, r1 - rb)
            r = rb + yb
            assert 0 <= ya < yb <= ny
            assert (rb + ya) * 2 + 1 < 2 * rows  # partial-sum slot of the piece
            starts.add(rb + ya)
            ring = np.full(PLANES * rw, np.nan)
            lat = src[j]

            def phase_a(q):
                y = ya - 1 + q
                y = y + ny if y < 0 else (y - ny if y >= ny else y)
                assert 0 <= y < ny
                xa = x[va]  # threads past the row do nothing
                g = np.stack([np.stack([lat[i, y, xa], lat[i, y, xa + 1]]) for i in range(9)])
                with np.errstate(invalid="ignore"):
                    c = collide(g.reshape(9, -1), omega).reshape(g.shape)
                for i in range(9):
                    base = strip_plane(i, q) * rw
                    assert 0 <= base and base + rw <= PLANES * rw
                    ring[base + xa], ring[base + xa + 1] = c[i, 0], c[i, 1]

            phase_a(0)
            phase_a(1)
            for y in range(ya, yb):
                q = y - ya + 1
                phase_a(q + 1)
                if race and q + 2 <= yb - ya + 1:
                    phase_a(q + 2)  # a thread already past this row's barrier
                rp, rz, rm = ((q - 1) & 3) * 3 * rw, (12 + (q % 3) * 3) * rw, (21 + ((q + 1) & 1) * 3) * rw
                pairs = {0: (rz + x, rz + x + 1), 1: (rz + rw + xl, rz + rw + x),
                         3: (rz + 2 * rw + xar, rz + 2 * rw + xbr), 2: (rp + x, rp + x + 1),
                         5: (rp + rw + xl, rp + rw + x), 6: (rp + 2 * rw + xar, rp + 2 * rw + xbr),
                         4: (rm + x, rm + x + 1), 7: (rm + rw + xar, rm + rw + xbr), 8: (rm + 2 * rw + xl, rm + 2 * rw + x)}
                g = np.stack([np.stack([ring[pairs[i][0][va]], ring[pairs[i][1][va]]]) for i in range(9)])
                assert not np.isnan(g[:, 0]).any(), "node a gathered a value no phase A wrote"
                assert not np.isnan(g[:, 1][:, vb[va]]).any(), "node b gathered a value no phase A wrote"
                with np.errstate(invalid="ignore"):
                    c = collide(g.reshape(9, -1), omega).reshape(g.shape)
                row = {-1: ny - 1 if y == 0 else y - 1, 0: y, 1: 0 if y == ny - 1 else y + 1}
                xa, bv = x[va], vb[va]
                for i in range(9):
                    ca = xa if CX[i] == 0 else (xar[va] if CX[i] > 0 else xl[va])
                    cb = (xa + 1 if CX[i] == 0 else (xbr[va] if CX[i] > 0 else xa))[bv]
                    assert (ca >= 0).all() and (ca < nx).all() and (cb >= 0).all() and (cb < nx).all()
                    dst[j][i, row[CY[i]], ca] = c[i, 0]
                    dst[j][i, row[CY[i]], cb] = c[i, 1][bv]
                    np.add.at(writes[j][i, row[CY[i]]], ca, 1)
                    np.add.at(writes[j][i, row[CY[i]]], cb, 1)
    for j, ny in enumerate(nys):
        assert (writes[j] == 1).all(), "every destination is written exactly once"
        assert np.array_equal(dst[j], two_plain_steps(src[j][:, :, :nx], omega))
        rb = int(row_base[j])
        # the last block of a sample adds the partial sums at these rows
        assert {rb + q for q in range(ny) if q == 0 or (rb + q) % per == 0} == {s for s in starts if rb <= s < rb + ny}


@pytest.mark.parametrize("nx,nys,grid", [(64, [5, 1, 2, 3, 7], 3), (64, [9, 9, 9], 2), (128, [4, 6], 5),
                                          (64, [2, 2, 2, 2], 16), (64, [30, 17, 1], 7), (63, [5, 3, 8], 4),
                                          (31, [7, 2], 3), (40, [6, 9], 2), (3, [4, 5], 2), (2, [3], 1), (97, [5], 2)])
@pytest.mark.parametrize("race", [False, True])
def test_strip_schedule_equals_two_plain_steps(nx, nys, grid, race):
    launch(nx, nys, grid, race, seed=nx + grid)
