"""The cluster kernel's data layout and in-place steps, replayed on the CPU (no GPU): a channel
sample's columns split into C slabs of cw columns, each block holding its slab's state once in shared
memory, row after row, each row the nine populations of CW >= cw columns (CW the smallest of 16, 32,
48, 64 that holds cw and fits, else cw; slot (i, y, lx) at y RW + i CW + lx, with the row stride RW >= 9 CW
padded so that rows start cw elements apart modulo the 32 banks).  The replay mirrors the kernel's index
arithmetic (the CUDA source is not imported): the
four node lists (boundary nodes, interior nodes at the slab's left and right edges, inner nodes),
placed by each thread's contiguous run and a scan, hold every fluid node exactly once, and the
warps' work units take every entry once; the link classes (wall, inlet, outlet, obstacle,
interior, in the kernel's order of tests); and one even and one odd step of the in-place order,
where each node reads and writes the same slots (so every slot of every fluid node is touched by
exactly one node per step, inside the block or in a neighbouring block at the right column), the
odd step gathers exactly the populations the two-lattice push of the even step would deliver, and
after the odd step the slots hold the next state in natural layout."""
import numpy as np
import pytest

from paper_2508_13867_gb300 import workloads as W
from paper_2508_13867_gb300 import uqlb as U
from paper_2508_13867_gb300.ensemble import sample_struct

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
INTERIOR, WALL, INLET, OUTLET, SOLID = 0, 1, 2, 3, 4
THREADS = 1024


def classify(solid, nx, ny, x, y):
    if y < 0 or y >= ny:
        return WALL
    if x < 0:
        return INLET
    if x >= nx:
        return OUTLET
    if solid[y, x]:
        return SOLID
    return INTERIOR


def replay(nd, csize, obstacle=True):
    spec = W.channel(nd, steps=10, steady_tol=0.0, obstacle=obstacle)
    solid = U.uqlb_obstacle_mask(sample_struct(spec)).astype(bool)
    nx, ny = spec.nx, spec.ny
    cw = (nx + csize - 1) // csize
    # row width: the smallest compiled width (16, 32, 48, 64) holding cw whose FP32 state (rows of
    # 9 W + 31 elements at most), link words and node list fit a block's shared memory, else cw itself;
    # on a compiled width the rows lie RW = 9 W + pad elements apart with RW = cw mod 32 (the banks)
    fits = lambda w: ((9 * w + 31) * ny * 4 + 15) // 16 * 16 + 2 * w * ny * 4 <= 227 * 1024 - 4096  # noqa: E731
    CW = next((w for w in (16, 32, 48, 64) if w >= cw and fits(w)), 0)
    RW = 9 * CW + (cw - 9 * CW) % 32 if CW else 9 * cw
    CW = CW or cw
    assert RW >= 9 * CW and (not CW > cw or RW % 32 == cw % 32)
    pl = ny * CW
    lists = []
    for rank in range(csize):
        x0 = rank * cw
        ncol = max(0, min(cw, nx - x0))
        nnodes = ny * ncol
        # link words: class of direction i in bits 3i..3i+2, bit 0 for a node at the slab's edge,
        # all ones for a solid node
        links = {}
        for y in range(ny):
            for lx in range(ncol):
                x = x0 + lx
                if solid[y, x]:
                    links[y, lx] = 0xFFFFFFFF
                    continue
                w = 0
                for i in range(1, 9):
                    w |= classify(solid, nx, ny, x + CX[i], y + CY[i]) << (3 * i)
                if lx == 0 or lx == ncol - 1:
                    w |= 1
                links[y, lx] = w
        # the lists (boundary, left edge, right edge, inner): contiguous runs of `chunk` nodes per
        # thread, placed by an exclusive scan
        def kind(w, lx):
            if w == 0xFFFFFFFF:
                return -1
            if w == 0:
                return 3
            return (1 if lx == 0 else 2) if (w == 1 and ncol > 1) else 0

        chunk = (nnodes + THREADS - 1) // THREADS
        runs = [range(min(nnodes, t * chunk), min(nnodes, t * chunk + chunk)) for t in range(THREADS)]
        lens = [0] * 4
        for run in runs:
            for n in run:
                k = kind(links[divmod(n, ncol)], n % ncol)
                if k >= 0:
                    lens[k] += 1
        base = [sum(lens[:c]) for c in range(4)]
        nlist = sum(lens)
        lst = [None] * nlist
        off = list(base)
        for run in runs:
            for n in run:
                y, lx = divmod(n, ncol)
                k = kind(links[y, lx], lx)
                if k >= 0:
                    assert lst[off[k]] is None
                    lst[off[k]] = (y, lx, k)
                    off[k] += 1
        # every fluid node listed once, in row-major order within each list
        fluid = [(y, lx) for y in range(ny) for lx in range(ncol) if not solid[y, x0 + lx]]
        assert sorted((y, lx) for y, lx, _ in lst) == fluid
        for k in range(4):
            part = lst[base[k]:base[k] + lens[k]]
            assert all(kk == k for _, _, kk in part) and [(y, lx) for y, lx, _ in part] == sorted(
                (y, lx) for y, lx, _ in part)
        assert all(y < 1 << 16 and lx < 1 << 16 for y, lx, _ in lst)
        # the work units: warp w takes unit w in round 0 and unit 32 r + NW - 1 - w in round r >= 1,
        # lane l its entry l; every entry is taken exactly once
        nw = THREADS // 32
        taken = np.zeros(nlist, int)
        r = 0
        while r * nw * 32 < nlist:
            for w in range(nw):
                for lane in range(32):
                    k = (r * nw + (w if r == 0 else nw - 1 - w)) * 32 + lane
                    if k < nlist:
                        taken[k] += 1
            r += 1
        assert (taken == 1).all()
        lists.append((x0, ncol, lst, base))
    # One even and one odd step of the in-place order, replayed symbolically on the slots of every
    # block ((rank, i, y, column) -> value).  A value ("g", x, y, i) is population i of the state the
    # run starts from; the collision of node (x, y) at step s makes ("post", s, x, y, i) of every
    # population, and a boundary link applies its rule: ("bc", s, x, y, i).
    slots = {}
    for rank in range(csize):
        x0, ncol, _, _ = lists[rank]
        for y in range(ny):
            for lx in range(ncol):
                for i in range(9):
                    slots[rank, i, y, lx] = ("g", x0 + lx, y, i)

    def block_of(x):
        return x // cw, x % cw

    def remote_slot(rank, to_left, i, y):
        # the kernel's remote(): column cw - 1 of the left block or column 0 of the right block
        return (rank - 1, i, y, cw - 1) if to_left else (rank + 1, i, y, 0)

    def link(x, y, i):
        return classify(solid, nx, ny, x + CX[i], y + CY[i])

    def step(s, odd):
        reads, writes = {}, {}
        for rank in range(csize):
            x0, ncol, lst, base = lists[rank]
            e0, e1, e2 = base[1], base[2], base[3]
            for k, (y, lx, kind) in enumerate(lst):
                x = x0 + lx
                own = (rank, 0, y, lx)
                src = [own]
                if not odd:
                    src += [(rank, i, y, lx) for i in range(1, 9)]
                else:
                    for i in range(1, 9):
                        sl = lx - CX[i]
                        if link(x, y, OPP[i]) != INTERIOR:
                            src.append((rank, i, y, lx))
                        elif 0 <= sl < ncol:
                            src.append((rank, OPP[i], y - CY[i], sl))
                        else:
                            assert kind in (0, 1, 2)  # remote reads only on the edge and boundary paths
                            r = remote_slot(rank, sl < 0, OPP[i], y - CY[i])
                            assert r[0] * cw + r[3] == x - CX[i]
                            src.append(r)
                for sl_ in src:
                    reads[sl_] = reads.get(sl_, 0) + 1
                dst = [own]
                for i in range(1, 9):
                    c = link(x, y, i)
                    if kind >= 1:
                        assert c == INTERIOR
                    if not odd or c != INTERIOR:
                        dst.append((rank, OPP[i], y, lx))
                    else:
                        dl = lx + CX[i]
                        if 0 <= dl < ncol:
                            dst.append((rank, i, y + CY[i], dl))
                        else:
                            assert kind in (0, 1, 2)
                            r = remote_slot(rank, dl < 0, i, y + CY[i])
                            assert r[0] * cw + r[3] == x + CX[i]
                            dst.append(r)
                # a node reads and writes the same slots within a step
                assert sorted(src) == sorted(dst), (s, odd, rank, y, lx)
                for d in dst:
                    writes[d] = writes.get(d, 0) + 1
                vals = [slots[q] for q in src]
                out = [None] * 9
                out[0] = ("post", s, x, y, 0)
                for i in range(1, 9):
                    c = link(x, y, i)
                    out[i] = ("post", s, x, y, i) if (c == INTERIOR or c in (WALL, SOLID)) else ("bc", s, x, y, i)
                yield (rank, x, y, lx, vals, dst, out)
        assert all(v == 1 for v in reads.values()) and all(v == 1 for v in writes.values())

    def incoming(s, x, y, i):
        # the population i that node (x, y) takes in after step s (the two-lattice push of step s)
        if i == 0:
            return ("post", s, x, y, 0)
        if link(x, y, OPP[i]) == INTERIOR:
            return ("post", s, x - CX[i], y - CY[i], i)
        c = link(x, y, OPP[i])
        return ("post", s, x, y, OPP[i]) if c in (WALL, SOLID) else ("bc", s, x, y, OPP[i])

    # even step 0: every node reads its own slots in natural order
    updates = list(step(0, False))
    for rank, x, y, lx, vals, dst, out in updates:
        assert vals == [("g", x, y, i) for i in range(9)]
    for rank, x, y, lx, vals, dst, out in updates:
        # writes go to the own slots opp(i) in the order of dst: slot 0 first, then opp(1) .. opp(8)
        slots[dst[0]] = out[0]
        for i in range(1, 9):
            slots[dst[i]] = out[i]
    # odd step 1: the gathered values are the two-lattice scheme's incoming populations after step 0
    updates = list(step(1, True))
    for rank, x, y, lx, vals, dst, out in updates:
        assert vals[0] == incoming(0, x, y, 0)
        for i in range(1, 9):
            assert vals[i] == incoming(0, x, y, i), (x, y, i)
    for rank, x, y, lx, vals, dst, out in updates:
        slots[dst[0]] = out[0]
        for i in range(1, 9):
            slots[dst[i]] = out[i]
    # after the odd step the state is in natural layout again: slot i of each node holds its
    # incoming population i of step 1
    for rank in range(csize):
        x0, ncol, lst, _ = lists[rank]
        for y, lx, _ in lst:
            for i in range(9):
                assert slots[rank, i, y, lx] == incoming(1, x0 + lx, y, i), (rank, y, lx, i)
    # the linear slot index of every slot a block holds stays inside its state and is one to one
    lin = {(i, y, lx): y * RW + i * CW + lx for i in range(9) for y in range(ny) for lx in range(cw)}
    assert len(set(lin.values())) == len(lin) and 0 <= min(lin.values()) and max(lin.values()) < RW * ny
    smem = (RW * ny * 4 + 15) // 16 * 16 + 2 * pl * 4
    return cw, smem


@pytest.mark.parametrize("nd,csize", [(4, 2), (5, 4), (6, 3), (20, 16), (7, 8), (5, 2), (5, 1)])
def test_cluster_push_writes_every_slot_once(nd, csize):
    cw, smem = replay(nd, csize)
    if nd == 20 and csize == 16:
        # the bench's cylinder: 28 columns per block (rows of 32), the state in FP32 fits one block's
        # shared memory
        assert cw == 28 and smem <= 227 * 1024 - 4096


def test_cluster_push_without_obstacle():
    replay(5, 4, obstacle=False)
