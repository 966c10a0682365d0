"""Host logic of the node-sharded path (no GPU): the split of the q
quadrature nodes among ranks (the q shifted systems of eq. 4.2 are
independent, end of Section 4.3), the set-up's validation of a node range
and its smaller workspace, and the collective hook over a world-size-2 gloo
group (sum of the partial quadrature sums, rank 0's stopping flag to every
rank)."""
import ctypes
import datetime
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_nodes_covers_the_contour_once():
    import paper_1404_1768_gb300 as fg
    for q in (1, 2, 7, 16, 32, 33):
        for world in range(1, min(q, 8) + 1):
            rs = [fg.shard_nodes(q, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == q
            for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in rs]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        fg.shard_nodes(4, 5, 0)


def _opts(fg, m0, j0, j1, coll, buf):
    o = fg.Options(m0, 1, 1e-12, 1e-3, 50, 1, 5, 1e-14, None, 0, 0)
    o.node_begin, o.node_end = j0, j1
    if coll is not None:
        o.collective = coll
    o.collective_buf = buf
    return o


def test_node_range_validation_and_workspace():
    """A context owning half the nodes needs about half the factor memory;
    ranges outside [0, q), empty ranges, and ranges without a collective
    hook or an aligned collective buffer are refused (FEAST_EINVAL)."""
    import paper_1404_1768_gb300 as fg
    lib = fg.load()
    n, m0, q = 1024, 64, 32
    p = fg.Pencil(0, n, 1, 1, n, 0, 0, 0)
    c = fg.Contour(0, 0.0, 0.0, 1.0, 1.0, q, 0)
    hook = fg.COLLECTIVE_FN(lambda *a: 0)

    def size(o):
        nb = ctypes.c_size_t(0)
        st = lib.feast_workspace_size(ctypes.byref(p), ctypes.byref(c), ctypes.byref(o), ctypes.byref(nb))
        return st, nb.value

    st, full = size(_opts(fg, m0, 0, 0, None, None))
    assert st == 0
    st, half = size(_opts(fg, m0, 0, 16, hook, 4096))
    assert st == 0
    # the complex64 factors (8 n^2 bytes per node) dominate what is saved
    assert full - half >= 16 * 8 * n * n
    assert half < 0.6 * full
    for j0, j1, h, b in ((-1, 4, hook, 4096), (4, 4, hook, 4096), (30, 33, hook, 4096),
                         (0, 16, None, 4096), (0, 16, hook, None), (0, 16, hook, 4096 + 8)):
        assert size(_opts(fg, m0, j0, j1, h, b))[0] == -1, (j0, j1)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    import paper_1404_1768_gb300 as fg
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=180))
    fn = fg.dist_collective()
    buf = torch.arange(6, dtype=torch.float64) * (rank + 1)
    fn(fg.FEAST_COLL_SUM, buf, 0)
    flag = torch.tensor([float(rank + 5)], dtype=torch.float64)
    fn(fg.FEAST_COLL_BCAST, flag, 0)
    out[rank] = (buf.tolist(), flag.item())
    dist.destroy_process_group()


def test_collective_hook_over_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29700 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.daemon = True
        pr.start()
    for pr in procs:
        pr.join(120)
    for pr in procs:
        if pr.is_alive():
            pr.terminate()
    assert [pr.exitcode for pr in procs] == [0, 0]
    for r in range(2):
        s, f = out[r]
        assert s == [3.0 * i for i in range(6)]     # (1 + 2) * i on both ranks
        assert f == 5.0                             # rank 0's value everywhere
