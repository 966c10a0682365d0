"""bench.py's roofline bookkeeping (host logic, no GPU): one entry per phase
of a pass, the dominant phase first, every entry with the keys the JSON line
promises and achieved / peak = frac."""
import argparse

import bench
from paper_1404_1768_gb300 import inputs

KEYS = {"bound", "achieved", "peak", "unit", "frac", "traffic", "phase", "share_of_pass"}


def _infos(warm):
    base = dict(qz_sweeps=300, qz_phases=0 if warm else 5000, qz_warm=int(warm), qz_rows=60 if warm else 64,
                qz_warm_resid=1e-14 if warm else 0.0, qz_warm_k=4 if warm else -1, refine_sweeps_max=0,
                ms_qz=5.0)
    return [dict(base) for _ in range(3)]


def test_dense_precision_form_rows():
    prob = bench.Problem(inputs.WORKLOADS["dense_n200_m64_q16"])
    args = argparse.Namespace(prec="c64r")
    ph = dict(ms_proj=1.0, ms_qz=5.0, ms_solve=2.0, ms_qr=3.0, ms_refine=0.0)
    for warm in (True, False):
        dom, others = bench.roofline_dominant(prob, args, ph, _infos(warm))
        assert dom["phase"] == "projected eigensolve"
        rows = [dom] + others
        assert {r["phase"] for r in rows} == {"projected eigensolve", "subspace-build solves",
                                             "orthonormalisation", "projection"}
        for r in rows:
            assert KEYS <= set(r)
            assert r["bound"] in ("hbm", "tensor", "alu")
            assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12 * max(1.0, r["frac"])
        assert abs(sum(r["share_of_pass"] for r in rows) - 1.0) < 1e-12


def test_band_rows():
    prob = bench.Problem(dict(inputs.WORKLOADS["band_n16384_m64_q16"], nx=12, m0=12))
    args = argparse.Namespace(prec="fp64")
    ph = dict(ms_proj=1.0, ms_qz=2.0, ms_solve=9.0, ms_qr=1.0, ms_refine=0.0)
    dom, others = bench.roofline_dominant(prob, args, ph, _infos(False))
    assert dom["phase"] == "subspace-build solves" and dom["bound"] == "alu"
    assert KEYS <= set(dom)


def test_warm_products_roofline_uses_the_library_events():
    """With the warm solve's own segment timing in the pass reports, the
    projected-eigensolve entry is that kernel's rate: total algorithmic
    flops / total segment time over the timed passes."""
    prob = bench.Problem(inputs.WORKLOADS["dense_n200_m64_q16"])
    args = argparse.Namespace(prec="c64r")
    ph = dict(ms_proj=1.0, ms_qz=5.0, ms_solve=2.0, ms_qr=3.0, ms_refine=0.0)
    infos = _infos(True)
    for i, inf in enumerate(infos):
        inf.update(ms_warm_gemm=2.0 + i, warm_gemm_flop=3.0e9)
    dom, _ = bench.roofline_dominant(prob, args, ph, infos)
    assert dom["phase"] == "projected eigensolve"
    expect = 9.0e9 / (9.0 / 1e3) / 1e12
    assert abs(dom["achieved"] - expect) < 1e-12 * expect
    assert abs(dom["kernel_ms_per_pass"] - 3.0) < 1e-12
    assert abs(dom["frac"] - dom["achieved"] / dom["peak"]) < 1e-12


def test_every_workload_has_an_arm_and_a_reference():
    """Each named workload dispatches to a GPU arm (or the dense/banded pass)
    and its kind is one the reference arm knows."""
    for name, cfg in inputs.WORKLOADS.items():
        arm = bench.arm_for(cfg)
        if arm is None:
            assert "nx" in cfg or "n" in cfg, name
            bench.Problem(dict(cfg, **({"nx": 24, "m0": 4} if "nx" in cfg else {"n": 40, "m0": 8})))
        else:
            assert callable(arm), name


def test_oracle_sample_scales_every_term_cubically():
    """The bounded oracle sample of the n = 4096 workload is the same
    generator at n/4, m0/4 (same q), and its pass time is scaled by 4^3;
    small dense and banded workloads are sampled as they are."""
    prob = bench.Problem.__new__(bench.Problem)
    prob.cfg = dict(inputs.WORKLOADS["dense_n4096_m1280_q32"], n=4096, m0=1280)
    prob.band, prob.n, prob.m0, prob.q = False, 4096, 1280, 32
    # (construct the sample's size only: the generator is not run here)
    s = 1
    while (prob.n / s) ** 2 * (prob.m0 / s) * prob.q > bench.ORACLE_PASS_WORK:
        s *= 2
    assert s == 4
    small = bench.Problem(inputs.WORKLOADS["dense_n200_m64_q16"])
    sp, sc = bench.oracle_sample(small)
    assert sp is small and sc == 1


def test_golden_oracle_run_parser_and_matching(tmp_path, monkeypatch):
    """The stored oracle run is read back as written (eigenvalues, counts,
    timings) and matched as a multiset: a permuted copy with one value moved
    by 1e-9 relative shows exactly that error and the count."""
    lam = [complex(0.5, -0.25), complex(-0.1, 0.7), complex(0.3, 0.3)]
    gdir = tmp_path / "tests" / "golden"
    gdir.mkdir(parents=True)
    lines = ["# header", "host Some CPU", "threads 8", "setup_s 12.5",
             "pass 1 0 2 0.000000e+00 40.0", "pass 2 3 1 1.0e-11 41.0",
             "flag 1", "k 2", "count 3", "exact_count 3", "err 1.0e-11"]
    lines += [f"eig {x.real:.17e} {x.imag:.17e} 1.0e-12" for x in lam]
    (gdir / "wl_oracle.txt").write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    g = bench.golden_oracle_run("wl")
    assert g["count"] == 3 and g["flag"] == 1 and g["k"] == 2 and g["threads"] == 8
    assert [p["s"] for p in g["passes"]] == [40.0, 41.0]
    assert list(g["lam"]) == lam
    got = {"lam": [lam[2], lam[0] * (1 + 1e-9), lam[1]], "count": 3}
    rep = bench.oracle_parity(got, g, 2)
    assert rep["count_match"] and rep["within_1e-8"]
    assert abs(rep["max_rel_eig_err_vs_oracle"] - 1e-9) < 1e-12
    got["lam"][1] = lam[0] * (1 + 1e-7)
    assert not bench.oracle_parity(got, g, 2)["within_1e-8"]
    assert bench.golden_oracle_run("absent") is None


def test_batch_schedule_autotuner_picks_the_fastest_trial():
    """The ragged batch's schedule autotuner times each candidate worker
    count once, in order, then keeps the fastest."""
    import paper_1404_1768_gb300 as fg
    t = fg.BatchSchedule(candidates=(16, 32, 64))
    seen = []
    for secs in (40.0, 30.0, 35.0):
        nw = t.next()
        seen.append(nw)
        t.record(nw, secs)
    assert seen == [16, 32, 64]
    assert t.best == 32 and t.next() == 32
    t.record(32, 50.0)            # a slower repeat keeps the best time
    assert t.times[32] == 30.0 and t.best == 32


def test_solve_step_runs_a_solve_again_after_a_bounded_wait_gave_up():
    """A solve that ends with ETIMEOUT (a bounded device wait gave up; the
    kernels returned and the context is intact) is run once more and listed
    in the JSON line's retried_solves; any other failure propagates."""
    import types

    class FeastError(RuntimeError):
        def __init__(self, status):
            super().__init__(f"status {status}")
            self.status = status

    fg = types.SimpleNamespace(FeastError=FeastError)
    calls = []

    def fake_solve_once(fg_, *a, **kw):
        calls.append(1)
        if len(calls) == 1:
            raise FeastError(-6)
        return {"ok": True}

    saved = bench.solve_once
    bench.RETRIES.clear()
    try:
        bench.solve_once = fake_solve_once
        assert bench.solve_step(fg, step="timed 0") == {"ok": True}
        assert len(calls) == 2
        assert len(bench.RETRIES) == 1 and bench.RETRIES[0]["step"] == "timed 0"

        def failing(fg_, *a, **kw):
            raise FeastError(-4)

        bench.solve_once = failing
        try:
            bench.solve_step(fg, step="timed 1")
            raise AssertionError("a singular pencil must not be retried")
        except FeastError as e:
            assert e.status == -4
        assert len(bench.RETRIES) == 1
    finally:
        bench.solve_once = saved
        bench.RETRIES.clear()
