"""The three-step row-strip kernel's schedule, replayed on the CPU.  Its ring-slot formula (3 / 2 / 1
slots for the c_y = +1 / 0 / -1 groups in each of its two rings), the pipeline of every piece
(phase A: row y + 2 at step t into ring 1; phase B: row y + 1 at step t + 1 from ring 1 into ring 2;
phase C: row y at step t + 2 from ring 2, pushed), its shorter last launches (two steps: phases A
and B with B pushing; one step: collide and push), the gather and push columns and the split of the
running rows into block ranges are mirrored here (the CUDA source is not imported).  Every ring value
carries the row it belongs to, and each gather checks that the slot it reads still holds the row it
expects (no slot is reused too early); every access is checked against its buffer; each destination
is written exactly once; one launch equals three (two, one) plain collide-and-stream steps.  The
kernel separates the phases of an iteration by two barriers, so a fast thread can run the next
iteration's phase A while slower threads are still in phase C: the replay also runs them in that
order."""
import numpy as np
import pytest

from tests.test_strip_schedule import CX, CY, collide

PLANES = 18


def plain_steps(f, omega, n):
    for _ in range(n):
        c = collide(f.reshape(9, -1), omega).reshape(f.shape)
        f = np.stack([np.roll(np.roll(c[i], CY[i], 0), CX[i], 1) for i in range(9)])
    return f


def ring3_plane(i, q):
    """Ring plane of direction i for the row with ring index q."""
    group, k = {2: (0, 0), 5: (0, 1), 6: (0, 2), 0: (1, 0), 1: (1, 1), 3: (1, 2), 4: (2, 0), 7: (2, 1),
                8: (2, 2)}[i]
    if group == 0:
        return (q % 3) * 3 + k
    if group == 1:
        return 9 + (q & 1) * 3 + k
    return 15 + k


def launch(nx, nys, steps_left, grid, race, seed):
    rng = np.random.default_rng(seed)
    omega = 1.3
    row_base = np.concatenate([[0], np.cumsum(nys)]).astype(int)
    rows = int(row_base[-1])
    np_ = ((nx + 1) // 2 + 31) // 32 * 32
    rw = 2 * np_
    src = []
    for ny in nys:
        a = np.full((9, ny, rw), np.nan)
        a[:, :, :nx] = rng.normal(0.0, 0.01, (9, ny, nx))
        src.append(a)
    dst = [np.full((9, ny, nx), np.nan) for ny in nys]
    writes = [np.zeros((9, ny, nx), int) for ny in nys]
    per = (rows + grid - 1) // grid
    x = 2 * np.arange(np_)
    va, vb = x < nx, x + 1 < nx
    xa, bv = x[va], vb[va]
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
            assert (rb + ya) * 3 + 2 < 3 * rows  # partial-sum slots of the piece
            n = steps_left[j]
            lat = src[j]
            rings = [np.full(PLANES * rw, np.nan), np.full(PLANES * rw, np.nan)]
            tags = [np.full(PLANES * rw, -10 ** 6), np.full(PLANES * rw, -10 ** 6)]

            def wrap(y):
                for _ in range(2):
                    y = y + ny if y < 0 else y
                for _ in range(2):
                    y = y - ny if y >= ny else y
                return y

            def put(k, y, g):
                q = y - ya + 4
                assert q >= 0
                for i in range(9):
                    base = ring3_plane(i, q) * rw
                    assert 0 <= base and base + rw <= PLANES * rw
                    rings[k][base + xa], rings[k][base + xa + 1] = g[i, 0], g[i, 1]
                    tags[k][base + xa], tags[k][base + xa + 1] = y, y

            def gather(k, y):
                q = y - ya + 4
                rp, rz, rm = ring3_plane(2, q - 1) * rw, ring3_plane(0, q) * rw, ring3_plane(4, q + 1) * rw
                pairs = {0: (rz + x, rz + x + 1), 1: (rz + rw + xl, rz + rw + x),
                         3: (rz + 2 * rw + xar, rz + 2 * rw + xbr), 2: (rp + x, rp + x + 1),
                         5: (rp + rw + xl, rp + rw + x), 6: (rp + 2 * rw + xar, rp + 2 * rw + xbr),
                         4: (rm + x, rm + x + 1), 7: (rm + rw + xar, rm + rw + xbr),
                         8: (rm + 2 * rw + xl, rm + 2 * rw + x)}
                for i in range(9):
                    want = y - CY[i]
                    for idx in (pairs[i][0][va], pairs[i][1][va][bv]):
                        assert (tags[k][idx] == want).all(), ("slot reused before its read", i, y)
                g = np.stack([np.stack([rings[k][pairs[i][0][va]], rings[k][pairs[i][1][va]]]) for i in range(9)])
                assert not np.isnan(g[:, 0]).any() and not np.isnan(g[:, 1][:, bv]).any()
                with np.errstate(invalid="ignore"):
                    return collide(g.reshape(9, -1), omega).reshape(g.shape)

            def load_collide(y):
                yy = wrap(y)
                assert 0 <= yy < ny
                g = np.stack([np.stack([lat[i, yy, xa], lat[i, yy, xa + 1]]) for i in range(9)])
                with np.errstate(invalid="ignore"):
                    return collide(g.reshape(9, -1), omega).reshape(g.shape)

            def push(y, c):
                row = {-1: ny - 1 if y == 0 else y - 1, 0: y, 1: 0 if y == ny - 1 else y + 1}
                for i in range(9):
                    ca = xa if CX[i] == 0 else (xar[va] if CX[i] > 0 else xl[va])
                    cb = (xa + 1 if CX[i] == 0 else (xbr[va] if CX[i] > 0 else xa))[bv]
                    assert (ca >= 0).all() and (ca < nx).all() and (cb >= 0).all() and (cb < nx).all()
                    dst[j][i, row[CY[i]], ca] = c[i, 0]
                    dst[j][i, row[CY[i]], cb] = c[i, 1][bv]
                    np.add.at(writes[j][i, row[CY[i]]], ca, 1)
                    np.add.at(writes[j][i, row[CY[i]]], cb, 1)

            if n == 1:
                for y in range(ya, yb):
                    push(y, load_collide(y))
            elif n == 2:
                put(0, ya - 1, load_collide(ya - 1))
                for y in range(ya - 1, yb):
                    put(0, y + 1, load_collide(y + 1))
                    # barrier
                    if y >= ya:
                        push(y, gather(0, y))
                    # barrier
            else:
                put(0, ya - 2, load_collide(ya - 2))
                put(0, ya - 1, load_collide(ya - 1))
                pending_c = None
                for y in range(ya - 2, yb):
                    put(0, y + 2, load_collide(y + 2))  # phase A
                    if pending_c is not None:
                        push(*pending_c)  # a slow thread's phase C of the previous iteration
                        pending_c = None
                    # barrier
                    put(1, y + 1, gather(0, y + 1))  # phase B
                    # barrier
                    if y >= ya:
                        c = (y, gather(1, y))  # phase C
                        if race:
                            pending_c = c
                        else:
                            push(*c)
                if pending_c is not None:
                    push(*pending_c)
    for j, ny in enumerate(nys):
        assert (writes[j] == 1).all(), "every destination is written exactly once"
        assert np.array_equal(dst[j], plain_steps(src[j][:, :, :nx], omega, steps_left[j]))


@pytest.mark.parametrize("nx,nys,grid", [(64, [5, 1, 2, 3, 7], 3), (64, [9, 9, 9], 2), (128, [4, 6], 5),
                                          (64, [2, 2, 2, 2], 16), (64, [30, 17, 1], 7), (63, [5, 3, 8], 4),
                                          (31, [7, 2], 3), (40, [6, 9], 2), (3, [4, 5], 2), (2, [3], 1), (97, [5], 2)])
@pytest.mark.parametrize("race", [False, True])
def test_strip3_schedule_equals_three_plain_steps(nx, nys, grid, race):
    launch(nx, nys, [3] * len(nys), grid, race, seed=nx + grid)


@pytest.mark.parametrize("steps_left", [[1, 2, 3, 2, 1], [2, 2, 2, 2, 2], [3, 1, 1, 3, 2]])
def test_strip3_last_launches_take_two_and_one_steps(steps_left):
    launch(64, [5, 1, 2, 3, 7], steps_left, 3, False, seed=11)
    launch(31, [4, 3, 6, 2, 5], steps_left, 4, True, seed=12)
