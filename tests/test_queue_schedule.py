"""The task-queue step's schedule (lbm_queue_schedule), host arithmetic only: its neighbour
chunks against a brute-force pass over every site's in-plane stencil, and its ticket order
against the dependency of the step (psi of the next step at a site needs the collisions of the
sites around it in planes z - 1 .. z + 1): every task once, every input of a psi task at a
smaller ticket, each psi task at the place its lag gives."""
import numpy as np
import pytest

from paper_1909_12390_gb300 import lbm


def _brute_neighbours(nx, ny, ts):
    """Per chunk, the set of other chunks holding a periodic 8-neighbour of one of its sites."""
    y, x = np.mgrid[0:ny, 0:nx]
    own = (y * nx + x) // ts
    nch = -(-(nx * ny) // ts)
    out = [set() for _ in range(nch)]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            other = (((y + dy) % ny) * nx + (x + dx) % nx) // ts
            for a, b in set(zip(own.ravel().tolist(), other.ravel().tolist())):
                if a != b:
                    out[a].add(b)
    return out


@pytest.mark.parametrize("nx,ny,nz,chunk,lag", [
    (256, 256, 12, 0, 0),     # the library's chunk (512) and lag (6) on the workload's planes
    (16, 12, 10, 0, 0),       # one chunk per plane
    (33, 17, 5, 64, 1),       # ragged chunks that start mid-row
    (24, 24, 3, 100, 2),      # the shortest march
    (40, 36, 33, 128, 3),
    (7, 5, 9, 1, 1),          # one site per chunk
    (64, 16, 16, 256, 6),
])
def test_schedule_orders_every_input_of_a_psi_task_first(nx, ny, nz, chunk, lag):
    res = lbm.queue_schedule(nx, ny, nz, chunk, lag)
    assert res is not None
    nch, nbr, tasks = res
    ts = min(chunk if chunk > 0 else 512, nx * ny)
    lag = lag if lag > 0 else 6
    assert nch == -(-(nx * ny) // ts)
    brute = _brute_neighbours(nx, ny, ts)
    for c in range(nch):
        listed = [int(v) for v in nbr[c] if v >= 0]
        assert len(listed) == len(set(listed))
        assert set(listed) == brute[c], c
        assert all(v == -1 for v in nbr[c][len(listed):])
    ncol = nz * nch
    assert len(tasks) == 2 * ncol
    col = tasks[tasks >= 0]
    psi = -tasks[tasks < 0] - 1
    assert np.array_equal(col, np.arange(ncol))          # every collision once, in plane order
    assert np.array_equal(np.sort(psi), np.arange(ncol))  # every psi chunk once
    pos = np.empty(ncol, dtype=np.int64)
    pos[col] = np.flatnonzero(tasks >= 0)
    for p in np.flatnonzero(tasks < 0):
        q = -int(tasks[p]) - 1
        z, c = divmod(q, nch)
        for dz in (-1, 0, 1):
            zz = (z + dz) % nz
            for cc in {c} | brute[c]:
                assert pos[zz * nch + cc] < p, (z, c, zz, cc)
        # the march places psi of (z, c) right after the collision of (z + 1 + lag, c)
        if 1 <= z and z + 1 + lag <= nz - 1:
            assert tasks[p - 1] == (z + 1 + lag) * nch + c
    # plane 0's psi chunks close the order (they need plane nz - 1's collisions)
    assert np.array_equal(-tasks[-nch:] - 1, np.arange(nch))


@pytest.mark.parametrize("shape", [(16, 16, 2), (0, 8, 8), (8, 0, 8)])
def test_schedule_rejects_grids_it_does_not_serve(shape):
    assert lbm.queue_schedule(*shape) is None
