"""bench.py's roofline bookkeeping (host logic, no GPU): one entry per phase
of a pass, the dominant phase first, every entry with the keys the JSON line
promises and achieved / peak = frac."""
import argparse

import bench
from paper_1404_1768_gb300 import inputs

KEYS = {"bound", "achieved", "peak", "unit", "frac", "traffic", "phase", "share_of_pass"}


def _infos(warm):
    base = dict(qz_sweeps=300, qz_phases=0 if warm else 5000, qz_warm=int(warm), qz_rows=60 if warm else 64,
                qz_warm_resid=1e-14 if warm else 0.0, qz_warm_k=4 if warm else -1, refine_sweeps_max=0)
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
