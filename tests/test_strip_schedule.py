"""The row-strip two-step kernel's schedule, replayed on the CPU: its ring-slot formula, the
gather and push columns, the split of the running rows into one range per block, and the
partial-sum slots the last block adds.  The kernel's index arithmetic is mirrored here (the
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
    src = [rng.normal(0.0, 0.01, (9, ny, nx)) for ny in nys]
    dst = [np.full((9, ny, nx), np.nan) for ny in nys]
    writes = [np.zeros((9, ny, nx), int) for ny in nys]
    per = (rows + grid - 1) // grid
    starts = set()
    np_ = nx // 2
    x = 2 * np.arange(np_)
    xl = np.where(x == 0, nx - 1, x - 1)
    xr = np.where(x + 2 == nx, 0, x + 2)
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
            ring = np.full(PLANES * nx, np.nan)
            lat = src[j]

            def phase_a(q):
                y = ya - 1 + q
                y = y + ny if y < 0 else (y - ny if y >= ny else y)
                assert 0 <= y < ny
                g = np.stack([np.stack([lat[i, y, x], lat[i, y, x + 1]]) for i in range(9)])
                c = collide(g.reshape(9, -1), omega).reshape(g.shape)
                for i in range(9):
                    base = strip_plane(i, q) * nx
                    assert 0 <= base and base + nx <= PLANES * nx
                    ring[base + x], ring[base + x + 1] = c[i, 0], c[i, 1]

            phase_a(0)
            phase_a(1)
            for y in range(ya, yb):
                q = y - ya + 1
                phase_a(q + 1)
                if race and q + 2 <= yb - ya + 1:
                    phase_a(q + 2)  # a thread already past this row's barrier
                rp, rz, rm = ((q - 1) & 3) * 3 * nx, (12 + (q % 3) * 3) * nx, (21 + ((q + 1) & 1) * 3) * nx
                pairs = {0: (rz + x, rz + x + 1), 1: (rz + nx + xl, rz + nx + x), 3: (rz + 2 * nx + x + 1, rz + 2 * nx + xr),
                         2: (rp + x, rp + x + 1), 5: (rp + nx + xl, rp + nx + x), 6: (rp + 2 * nx + x + 1, rp + 2 * nx + xr),
                         4: (rm + x, rm + x + 1), 7: (rm + nx + x + 1, rm + nx + xr), 8: (rm + 2 * nx + xl, rm + 2 * nx + x)}
                g = np.stack([np.stack([ring[pairs[i][0]], ring[pairs[i][1]]]) for i in range(9)])
                assert not np.isnan(g).any(), "gathered a ring value no phase A wrote"
                c = collide(g.reshape(9, -1), omega).reshape(g.shape)
                row = {-1: ny - 1 if y == 0 else y - 1, 0: y, 1: 0 if y == ny - 1 else y + 1}
                for i in range(9):
                    ca = x if CX[i] == 0 else (x + 1 if CX[i] > 0 else xl)
                    cb = x + 1 if CX[i] == 0 else (xr if CX[i] > 0 else x)
                    assert (ca >= 0).all() and (ca < nx).all() and (cb >= 0).all() and (cb < nx).all()
                    dst[j][i, row[CY[i]], ca] = c[i, 0]
                    dst[j][i, row[CY[i]], cb] = c[i, 1]
                    np.add.at(writes[j][i, row[CY[i]]], ca, 1)
                    np.add.at(writes[j][i, row[CY[i]]], cb, 1)
    for j, ny in enumerate(nys):
        assert (writes[j] == 1).all(), "every destination is written exactly once"
        assert np.array_equal(dst[j], two_plain_steps(src[j], omega))
        rb = int(row_base[j])
        # the last block of a sample adds the partial sums at these rows
        assert {rb + q for q in range(ny) if q == 0 or (rb + q) % per == 0} == {s for s in starts if rb <= s < rb + ny}


@pytest.mark.parametrize("nx,nys,grid", [(64, [5, 1, 2, 3, 7], 3), (64, [9, 9, 9], 2), (128, [4, 6], 5),
                                          (64, [2, 2, 2, 2], 16), (64, [30, 17, 1], 7)])
@pytest.mark.parametrize("race", [False, True])
def test_strip_schedule_equals_two_plain_steps(nx, nys, grid, race):
    launch(nx, nys, grid, race, seed=nx + grid)
