"""The cluster kernel's data layout and push, replayed on the CPU (no GPU): a channel sample's
columns split into C slabs of cw columns, each block holding [9][ny][cw] twice in shared memory.
The replay mirrors the kernel's index arithmetic (the CUDA source is not imported): each thread's
division-free walk over its block's nodes visits every owned node exactly once; the link classes
(wall, inlet, outlet, obstacle, interior, in the kernel's order of tests); and the push of one step,
where every population of every fluid node lands in exactly one slot of the next state, inside the
block's buffer or its left or right neighbour's, and every slot of every fluid node is written
exactly once (by the neighbour it streams from or by its own node's boundary rule)."""
import numpy as np
import pytest

from paper_2508_13867_gb300 import workloads as W
from paper_2508_13867_gb300 import uqlb as U
from paper_2508_13867_gb300.ensemble import sample_struct

CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
INTERIOR, WALL, INLET, OUTLET, SOLID = 0, 1, 2, 3, 4
THREADS = 512


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
    pl = ny * cw
    writes = np.zeros((csize, 9, pl), int)
    for rank in range(csize):
        x0 = rank * cw
        ncol = max(0, min(cw, nx - x0))
        nnodes = ny * ncol
        visited = np.zeros(nnodes, int)
        walk_r, walk_c = (THREADS // ncol, THREADS % ncol) if ncol else (0, 0)
        for tid in range(THREADS):
            y, lx = (tid // ncol, tid % ncol) if ncol else (0, 0)
            for n in range(tid, nnodes, THREADS):
                assert (y, lx) == divmod(n, ncol), (rank, tid, n)
                visited[n] += 1
                x = x0 + lx
                if not solid[y, x]:
                    own = y * cw + lx
                    assert 0 <= own < pl
                    writes[rank, 0, own] += 1
                    for i in range(1, 9):
                        c = classify(solid, nx, ny, x + CX[i], y + CY[i])
                        if c == INTERIOR:
                            dl, dy = lx + CX[i], y + CY[i]
                            target, col = rank, dl
                            if dl < 0:
                                target, col = rank - 1, cw - 1
                            elif dl >= ncol:
                                target, col = rank + 1, 0
                            assert 0 <= target < csize and 0 <= col < cw and 0 <= dy < ny
                            # the destination node is the neighbour itself in that block's slab
                            assert target * cw + col == x + CX[i]
                            writes[target, i, dy * cw + col] += 1
                        else:
                            writes[rank, OPP[i], own] += 1
                lx += walk_c
                y += walk_r + (1 if lx >= ncol else 0)
                lx -= ncol if lx >= ncol else 0
        assert (visited == 1).all()
    for rank in range(csize):
        x0 = rank * cw
        ncol = max(0, min(cw, nx - x0))
        for y in range(ny):
            for lx in range(cw):
                fluid = lx < ncol and not solid[y, x0 + lx]
                assert (writes[rank, :, y * cw + lx] == (1 if fluid else 0)).all(), (rank, y, lx)
    smem = 2 * 9 * pl * 4 + pl * 4
    return cw, smem


@pytest.mark.parametrize("nd,csize", [(4, 2), (5, 4), (6, 3), (20, 16), (7, 8), (5, 1)])
def test_cluster_push_writes_every_slot_once(nd, csize):
    cw, smem = replay(nd, csize)
    if nd == 20 and csize == 16:
        # the bench's cylinder: 28 columns per block, both states in FP32 fit one block's shared memory
        assert cw == 28 and smem <= 227 * 1024 - 4096


def test_cluster_push_without_obstacle():
    replay(5, 4, obstacle=False)
