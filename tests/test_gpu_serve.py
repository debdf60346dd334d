"""Serving form: requests of different grids, eps/mu, precisions and end
times submitted while others run give the same results as when each runs
alone, match the oracle (FP64), and HBM-budget admission holds."""
import numpy as np
import pytest

import synth
from oracle import scheme
from tests.gpu_util import rel_l2, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
REQS = [
    dict(n=(16, 16, 16), eps=1.0, mu=1.0, prec="fp64", t_end=3.7, nsteps=1),
    dict(n=(24, 20, 12), eps=2.0, mu=0.5, prec="fp32", t_end=11.0, nsteps=1, hi=(2.0, 3.0, 2.5)),
    dict(n=(32, 32, 32), eps=1.3, mu=2.2, prec="fp32", t_end=25.0, nsteps=4, every=1),
    dict(n=(32, 32, 32), eps=3.1, mu=1.1, prec="fp64", t_end=1.5, nsteps=1),
    dict(n=(48, 64, 80), eps=1.7, mu=1.0, prec="fp32", t_end=49.0, nsteps=1),
    dict(n=(16, 16, 16), eps=1.0, mu=2.0, prec="fp64", t_end=7.0, nsteps=3, every=1),
    dict(n=(64, 64, 64), eps=2.5, mu=2.5, prec="fp64", t_end=9.0, nsteps=1),
    dict(n=(8, 12, 10), eps=1.1, mu=0.9, prec="fp32", t_end=30.0, nsteps=2, hi=(2.0, 3.0, 2.5)),
]


def _inputs(mx, spec, seed):
    import torch

    g = synth.Grid(spec["n"], (0, 0, 0), spec.get("hi", (TWO_PI,) * 3))
    E0, H0 = synth.random_divfree_fields(g, seed=seed, sigma=max(spec["n"]) / 5)
    dt = torch.float64 if spec["prec"] == "fp64" else torch.float32
    pin = lambda a: torch.tensor(a, dtype=dt).pin_memory()  # noqa: E731
    out = [torch.empty(E0.shape, dtype=dt).pin_memory() for _ in range(2)]
    return g, E0, H0, pin(E0), pin(H0), out[0], out[1]


def _submit(mx, srv, spec, bufs):
    g, _, _, E0p, H0p, Eo, Ho = bufs
    P = mx.MX_FP64 if spec["prec"] == "fp64" else mx.MX_FP32
    return srv.submit(spec["n"], E0p, H0p, Eo, Ho, spec["t_end"], spec["eps"], spec["mu"], P, spec["nsteps"],
                      spec.get("every", 0), lo=g.lo, hi=g.hi)


def test_serve_same_alone_and_in_mix():
    mx = solver_mod()
    bufs = [_inputs(mx, sp, 40 + i) for i, sp in enumerate(REQS)]
    srv = mx.Server(8 << 30, max_active=16)
    alone = []
    for sp, b in zip(REQS, bufs):
        rid = _submit(mx, srv, sp, b)
        assert srv.wait(rid) == 2
        inv, lat = srv.result(rid)
        alone.append((b[5].clone().double().numpy(), b[6].clone().double().numpy(), inv))
        assert lat > 0
    # all at once: they overlap on the device
    ids = [_submit(mx, srv, sp, b) for sp, b in zip(REQS, bufs)]
    for rid in ids:
        assert srv.wait(rid) == 2
    st = srv.stats()
    assert st["completed"] == 2 * len(REQS) and st["rejected"] == 0
    assert st["hbm_high_water"] <= st["hbm_budget"]
    assert st["pooled_contexts"] >= 1
    for i, (sp, b, rid) in enumerate(zip(REQS, bufs, ids)):
        inv, _ = srv.result(rid)
        np.testing.assert_array_equal(b[5].double().numpy(), alone[i][0])
        np.testing.assert_array_equal(b[6].double().numpy(), alone[i][1])
        assert len(inv) == len(alone[i][2])
        for ra, rb in zip(inv, alone[i][2]):
            for k in ra:
                np.testing.assert_array_equal(ra[k], rb[k])
        # against the oracle
        g, E0, H0 = b[0], b[1], b[2]
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, sp["eps"], sp["mu"], sp["t_end"])
        tol = 1e-12 if sp["prec"] == "fp64" else 1e-5
        assert rel_l2(alone[i][0], alone[i][1], Eo, Ho) < tol
        expect = 2 if sp.get("every", 0) == 0 else 1 + sp["nsteps"]
        assert len(inv) == expect
    srv.close()


def test_serve_budget_admission_and_rejection():
    mx = solver_mod()
    small = dict(n=(32, 32, 32), eps=1.0, mu=1.0, prec="fp32", t_end=2.0, nsteps=1)
    big = dict(n=(128, 128, 128), eps=1.0, mu=1.0, prec="fp64", t_end=2.0, nsteps=1)
    fp_small = mx.footprint_bytes(small["n"], mx.MX_FP32, mx.MX_FORM_SPECTRAL)
    fp_big = mx.footprint_bytes(big["n"], mx.MX_FP64, mx.MX_FORM_SPECTRAL)
    budget = int(2.5 * fp_small)  # two small requests fit, the big one never does
    assert fp_big > budget
    srv = mx.Server(budget, max_active=8)
    bs = [_inputs(mx, small, 60 + i) for i in range(6)]
    bb = _inputs(mx, big, 70)
    ids = [_submit(mx, srv, small, b) for b in bs[:3]]
    big_id = _submit(mx, srv, big, bb)
    ids += [_submit(mx, srv, small, b) for b in bs[3:]]
    for rid in ids:
        assert srv.wait(rid) == 2
    assert srv.wait(big_id) == -mx.MX_E_NOMEM
    st = srv.stats()
    assert st["completed"] == 6 and st["rejected"] == 1
    assert st["hbm_high_water"] <= budget
    for b, rid in zip(bs, ids):
        g, E0, H0 = b[0], b[1], b[2]
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, 2.0)
        assert rel_l2(b[5].double().numpy(), b[6].double().numpy(), Eo, Ho) < 1e-5
    srv.close()
