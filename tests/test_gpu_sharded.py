"""Node-sharded GFEAST (end of Section 4.3: the q shifted systems of eq. 4.2
are independent): two processes on the test GPU each own half of the
quadrature nodes -- their own shifted matrices, factors and solves -- and
combine their partial quadrature sums through a world-size-2 gloo group
(host copies of U).  Their first subspace must equal the one-rank run's, and
their runs must stop at the same pass with the same eigenvalues as the
one-rank run and the oracle.  (Unmeasured on multi-GPU hardware: every box
of this run has one GPU.)"""
import datetime
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # n = 200 workload, FP64, 16 trapezoid nodes
    "fp64_n200": dict(n=200, m0=64, seed=0, kw=dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-12)),
    # precision form at a width that takes the warm projected solve, the
    # Cholesky QR and the defect-form line 16
    "c64r_n640": dict(n=640, m0=208, seed=1, kw=dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-10,
                                                     prec=1, refine_tol=1e-13, max_refine=4)),
}


def _run(fg, p, kw, **extra):
    g = fg.Feast(p.A, p.B, p.Y, **kw, **extra)
    U1 = g.get("U1")
    hist = g.run()
    r = g.eigs(want_vectors=False)
    g.close()
    return U1, [h["flag"] for h in hist], r


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_1404_1768_gb300 as fg
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=180))
    c = CASES[case]
    p = inputs.prescribed_pencil(c["n"], c["m0"], seed=c["seed"])
    rng = fg.shard_nodes(c["kw"]["q"], world, rank)
    U1, flags, r = _run(fg, p, c["kw"], node_range=rng, collective=fg.dist_collective())
    out[rank] = dict(U1=U1, flags=flags, count=r["count"], flag=r["flag"], lam=r["lam"], res=r["res"])
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_ranks_sharing_the_nodes_match_one_rank(case):
    import oracle
    import paper_1404_1768_gb300 as fg
    c = CASES[case]
    p = inputs.prescribed_pencil(c["n"], c["m0"], seed=c["seed"])
    U1, flags, r1 = _run(fg, p, c["kw"])

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29800 + os.getpid() % 500 + (7 if case.startswith("c64") else 0)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, out)) for r in range(2)]
    for pr in procs:
        pr.daemon = True
        pr.start()
    for pr in procs:
        pr.join(600)
    for pr in procs:
        if pr.is_alive():
            pr.terminate()
    assert [pr.exitcode for pr in procs] == [0, 0]
    okw = {k: v for k, v in c["kw"].items() if k not in ("prec", "refine_tol", "max_refine")}
    o = oracle.Feast(p.A, p.B, p.Y, **okw)
    o.run()
    ro = o.result()
    o.close()
    lo = np.sort_complex(ro["lam"])
    for rank in range(2):
        w = out[rank]
        # the same first subspace (the node sums in another order)
        assert np.max(np.abs(w["U1"] - U1)) < 1e-11, rank
        # both ranks stop together, at the one-rank run's pass, with its flag
        assert w["flags"] == flags, (rank, w["flags"], flags)
        assert w["count"] == r1["count"] == ro["count"] == p.inside_count()
        ls = np.sort_complex(w["lam"])
        np.testing.assert_allclose(ls, np.sort_complex(r1["lam"]), rtol=0, atol=1e-10)
        tol = 1e-10 if "prec" not in c["kw"] else 1e-8
        np.testing.assert_allclose(ls, lo, rtol=0, atol=tol * max(1.0, np.abs(lo).max()))
        assert np.max(w["res"]) < 1e-10
