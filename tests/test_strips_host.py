"""Host-side logic of the x-strip decomposition (sim_strips_layout, no GPU
call): the partition of the columns, the halo each strip stores and the
positions it computes, and the halo exchange between neighbouring strips run
as two gloo ranks on the CPU, each holding one strip of a field and trading
its halo columns with the other by point-to-point messages."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1802_04243_gb300 as sim
from paper_1802_04243_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = sim.STRIP_HALO
G = 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sim.load()


@pytest.mark.parametrize("nx,n", [(8, 1), (16, 2), (37, 3), (128, 2), (128, 16), (1000, 7), (4864, 8), (4864, 64)])
def test_layout_tiles_the_columns_and_holds_the_halo(nx, n):
    lays = [sim.strips_layout(nx, n, k) for k in range(n)]
    assert lays[0]["own"][0] == 0 and lays[-1]["own"][1] == nx
    for k, lay in enumerate(lays):
        a, b = lay["own"]
        c0, c1 = lay["compute"]
        s0, s1 = lay["store"]
        assert b - a >= 2 * H                                   # a neighbour's halo lies inside its owner
        if k + 1 < n:
            assert lays[k + 1]["own"][0] == b
        # computed positions: the owned columns plus a halo on each side facing
        # another strip, start aligned to the 32-wide row segments
        assert c0 % 32 == 0 and c0 <= max(0, a - H)
        assert c1 == (nx + 1 if k == n - 1 else b + H)
        # stored columns: every stencil of a computed position (two columns
        # each way) stays inside the window; the whole problem's ghosts at
        # the ends
        assert (s0, s1) == (c0 - G, c1 + G)
        assert s0 >= -G and s1 <= nx + G + 1
    assert lays[0]["store"][0] == -G and lays[-1]["store"][1] == nx + G + 1


@pytest.mark.parametrize("nx,n", [(7, 1), (15, 2), (100, 13), (10_000, 65), (100, 0)])
def test_layout_rejects_strips_narrower_than_two_halos(nx, n):
    with pytest.raises(sim.SimError) as e:
        sim.strips_layout(nx, n, 0)
    assert e.value.status == sim.SIM_EINVAL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nx, ny, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1802_04243_gb300 as s
    rng = np.random.default_rng(3)
    whole = rng.standard_normal((ny + 2 * G + 1, nx + 2 * G + 1))     # one field over the extended grid
    lay = s.strips_layout(nx, world, rank)
    s0, s1 = lay["store"]
    a, b = lay["own"]
    col = lambda i: i + G                                             # column of the extended grid
    mine = np.full((whole.shape[0], s1 - s0), np.nan)
    # a strip starts with its owned columns (and the whole problem's ghost
    # columns at the domain ends) only
    lo = s0 if rank == 0 else a
    hi = s1 if rank == world - 1 else b
    mine[:, lo - s0:hi - s0] = whole[:, col(lo):col(hi)]
    # the exchange: across the boundary X with each neighbour, send the halo
    # the neighbour stores from the owned columns and receive the own halo
    if rank + 1 < world:
        X = b
        dist.send(torch.from_numpy(np.ascontiguousarray(mine[:, X - H - s0:X - s0])), dst=rank + 1)
        t = torch.empty((whole.shape[0], H), dtype=torch.float64)
        dist.recv(t, src=rank + 1)
        mine[:, X - s0:X + H - s0] = t.numpy()
    if rank > 0:
        X = a
        t = torch.empty((whole.shape[0], H), dtype=torch.float64)
        dist.recv(t, src=rank - 1)
        mine[:, X - H - s0:X - s0] = t.numpy()
        dist.send(torch.from_numpy(np.ascontiguousarray(mine[:, X - s0:X + H - s0])), dst=rank - 1)
    # after one exchange every column the strip's owned results depend on,
    # [own0 - halo, own1 + halo) within the window, holds the whole field's values
    need0, need1 = max(s0, a - H), min(s1, b + H)
    ok = np.array_equal(mine[:, need0 - s0:need1 - s0], whole[:, col(need0):col(need1)])
    out[rank] = (ok, (a, b), (s0, s1))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("nx", [64, 101])
def test_two_gloo_ranks_exchange_the_halos_of_their_strips(nx):
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), nx, 12, out), nprocs=world, join=True)
        res = dict(out)
    assert all(res[r][0] for r in range(world)), res
    assert res[0][1][1] == res[1][1][0]                   # adjacent owned ranges
