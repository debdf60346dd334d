"""Batched form: instances advanced together by one persistent launch agree
bit for bit with the same instance run alone, agree with a single-context
solve to round-off, and match the oracle field by field (FP64 and FP32)."""
import numpy as np
import pytest

import synth
from oracle import scheme
from tests.gpu_util import field_rel_l2, inv_diff, inv_scales, rel_l2, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
SPECS = [
    dict(n=(32, 32, 32), eps=1.5, mu=2.5, h=0.031),
    dict(n=(48, 64, 80), eps=3.2, mu=1.1, h=0.017),
    dict(n=(64, 64, 64), eps=1.0, mu=4.0, h=0.09),
    dict(n=(24, 20, 12), lo=(0, 0, 0), hi=(2.0, 3.0, 2.5), eps=2.0, mu=1.0, h=0.05),  # direct coefficients
    dict(n=(6, 10, 4), eps=1.2, mu=1.3, h=0.2),  # odd Mx, tiny
]


def _run_batch(mx, specs, prec, steps, every):
    import torch

    b = mx.Batch(specs, prec)
    b.load_random(100, 3.0)
    b.step(steps, every)
    b.step(steps, every)  # second call replays the captured graph
    b.sync()
    out = []
    dt = torch.float64 if prec == mx.MX_FP64 else torch.float32
    for i, sp in enumerate(specs):
        inst = b.instance(i)
        nx, ny, nz = sp["n"]
        E = torch.empty((3, nz, ny, nx), dtype=dt, device="cuda")
        H = torch.empty_like(E)
        inst.read(E, H)
        inst.sync()
        out.append((E.double().cpu().numpy(), H.double().cpu().numpy(), inst.invariants(), inst.time()))
    used = b.graph_used()
    b.close()
    return out, used


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_alone_equals_in_mix_and_single_context(prec):
    import torch

    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    steps, every = 7, 2
    mix, used = _run_batch(mx, SPECS, P, steps, every)
    assert used == 1, f"graph capture refused: CUDA error {-used}"
    tol = 1e-12 if prec == "fp64" else 1e-6
    for i, sp in enumerate(SPECS):
        # the same instance alone in a batch (seed of instance i is 100 + i: pass it as seed)
        b = mx.Batch([sp], P)
        b.instance(0).load_random(100 + i, 3.0)
        b.step(steps, every)
        b.step(steps, every)
        b.sync()
        inst = b.instance(0)
        nx, ny, nz = sp["n"]
        dt = torch.float64 if P == mx.MX_FP64 else torch.float32
        E = torch.empty((3, nz, ny, nx), dtype=dt, device="cuda")
        H = torch.empty_like(E)
        inst.read(E, H)
        inst.sync()
        alone = (E.double().cpu().numpy(), H.double().cpu().numpy(), inst.invariants())
        b.close()
        np.testing.assert_array_equal(mix[i][0], alone[0])
        np.testing.assert_array_equal(mix[i][1], alone[1])
        assert len(mix[i][2]) == len(alone[2]) == 1 + 2 * steps // every
        for ra, rb in zip(mix[i][2], alone[2]):
            for k in ra:
                np.testing.assert_array_equal(ra[k], rb[k])
        t, nstep = mix[i][3]
        assert nstep == 2 * steps and abs(t - 2 * steps * sp["h"]) < 1e-12
        # a single spectral-form context from the same initial state
        lo = sp.get("lo", (0, 0, 0))
        hi = sp.get("hi", (TWO_PI,) * 3)
        s = mx.Solver(sp["n"], lo, hi, sp["eps"], sp["mu"], P, mx.MX_FORM_SPECTRAL)
        s.load_random(100 + i, 3.0)
        s.step(sp["h"], 2 * steps, every)
        Es, Hs = torch.empty_like(E), torch.empty_like(H)
        s.read(Es, Hs)
        s.sync()
        inv_s = s.invariants()
        s.close()
        assert rel_l2(mix[i][0], mix[i][1], Es.double().cpu().numpy(), Hs.double().cpu().numpy()) < tol
        sc = inv_scales(inv_s[0], sp["eps"], sp["mu"])
        for ra, rb in zip(mix[i][2], inv_s):
            assert ra["step"] == rb["step"]
            assert inv_diff(ra, rb, sc) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_per_field(prec):
    """Every instance of a mixed batch against the oracle (one step of size 9 h), each of the six
    fields within 1e-12 (FP64) or 1e-5 (FP32) relative L2, invariants of the last record within
    the same tolerance of the oracle's physical-space values."""
    from oracle import invariants as oinv

    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    npdt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    specs = [SPECS[3], SPECS[4], dict(n=(16, 12, 8), eps=1.7, mu=0.6, h=0.043),
             dict(n=(32, 24, 40), eps=2.5, mu=1.5, h=0.071)]
    b = mx.Batch(specs, P)
    inits = []
    for i, sp in enumerate(specs):
        g = synth.Grid(sp["n"], sp.get("lo", (0, 0, 0)), sp.get("hi", (TWO_PI,) * 3))
        rng = np.random.default_rng(30 + i)
        E0 = rng.standard_normal((3,) + g.shape).astype(npdt).astype(np.float64)
        H0 = rng.standard_normal((3,) + g.shape).astype(npdt).astype(np.float64)
        b.instance(i).load(E0.astype(npdt), H0.astype(npdt))
        inits.append((g, E0, H0))
    b.step(9, 3)
    b.sync()
    for i, sp in enumerate(specs):
        g, E0, H0 = inits[i]
        inst = b.instance(i)
        E, H = inst.read_numpy()
        Eo, Ho = scheme.solve(E0, H0, g.lo, g.hi, sp["eps"], sp["mu"], 9 * sp["h"])
        errs = field_rel_l2(E.astype(np.float64), H.astype(np.float64), Eo, Ho)
        assert max(errs) < tol, (i, errs)
        inv = inst.invariants()
        assert len(inv) == 4
        r0 = oinv.invariants(E0, H0, g.lo, g.hi, sp["eps"], sp["mu"])
        rn = oinv.invariants(Eo, Ho, g.lo, g.hi, sp["eps"], sp["mu"])
        sc = inv_scales(r0, sp["eps"], sp["mu"])
        assert inv_diff(inv[-1], rn, sc) < tol
    b.close()


def _run_literal_batch(mx, specs, prec, inits, steps, every, calls=2, form=None):
    import torch

    b = mx.Batch(specs, prec, form=mx.MX_FORM_LITERAL if form is None else form)
    npdt = np.float64 if prec == mx.MX_FP64 else np.float32
    for i, (E0, H0) in enumerate(inits):
        b.instance(i).load(E0.astype(npdt), H0.astype(npdt))
    for _ in range(calls):
        b.step(steps, every)  # the second call replays the captured graph
    b.sync()
    out = []
    for i in range(len(specs)):
        inst = b.instance(i)
        E, H = inst.read_numpy()
        out.append((E.astype(np.float64), H.astype(np.float64), inst.invariants(), inst.time()))
    used = b.graph_used()
    b.close()
    return out, used


@pytest.mark.parametrize("form", ["literal", "xy"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_literal_batch_alone_equals_in_mix_and_matches_oracle(prec, form):
    """Literal-form batch (every instance's x, y, fused z, y, x passes as parallel graph branches, with
    its shape's autotuned schedules): bit-identical alone and in the mix, each of the six fields
    against the oracle's literal stepping (Alg. 1 + Alg. 2 with t_end = h, repeated) within 1e-12
    (FP64) or 1e-5 (FP32), invariants of the last record against the oracle's."""
    from oracle import invariants as oinv

    mx = solver_mod()
    P = mx.MX_FP64 if prec == "fp64" else mx.MX_FP32
    npdt = np.float64 if prec == "fp64" else np.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    F = mx.MX_FORM_LITERAL if form == "literal" else mx.MX_FORM_XY
    if form == "literal":
        specs = [SPECS[3], SPECS[4], dict(n=(16, 12, 32), eps=1.7, mu=0.6, h=0.043),
                 dict(n=(20, 24, 80), eps=2.2, mu=1.4, h=0.03)]
    else:  # the xy-resident form needs fused plans for nz (FP64: 2^a)
        specs = [dict(n=(24, 20, 16), lo=(0, 0, 0), hi=(2.0, 3.0, 2.5), eps=2.0, mu=1.0, h=0.05), SPECS[4],
                 dict(n=(16, 12, 32), eps=1.7, mu=0.6, h=0.043), dict(n=(20, 24, 64), eps=2.2, mu=1.4, h=0.03)]
    inits = []
    for i, sp in enumerate(specs):
        g = synth.Grid(sp["n"], sp.get("lo", (0, 0, 0)), sp.get("hi", (TWO_PI,) * 3))
        rng = np.random.default_rng(60 + i)
        inits.append((rng.standard_normal((3,) + g.shape).astype(npdt).astype(np.float64),
                      rng.standard_normal((3,) + g.shape).astype(npdt).astype(np.float64)))
    steps, every = 3, 1
    mix, used = _run_literal_batch(mx, specs, P, inits, steps, every, form=F)
    assert used == 1, f"graph capture refused: CUDA error {-used}"
    for i, sp in enumerate(specs):
        alone, _ = _run_literal_batch(mx, [sp], P, [inits[i]], steps, every, form=F)
        np.testing.assert_array_equal(mix[i][0], alone[0][0])
        np.testing.assert_array_equal(mix[i][1], alone[0][1])
        assert len(mix[i][2]) == len(alone[0][2]) == 1 + 2 * steps
        for ra, rb in zip(mix[i][2], alone[0][2]):
            for k in ra:
                np.testing.assert_array_equal(ra[k], rb[k])
        t, nstep = mix[i][3]
        assert nstep == 2 * steps and abs(t - 2 * steps * sp["h"]) < 1e-12
        g = synth.Grid(sp["n"], sp.get("lo", (0, 0, 0)), sp.get("hi", (TWO_PI,) * 3))
        E0, H0 = inits[i]
        Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, sp["eps"], sp["mu"], sp["h"], 2 * steps)
        errs = field_rel_l2(mix[i][0], mix[i][1], Eo, Ho)
        assert max(errs) < tol, (i, errs)
        r0 = oinv.invariants(E0, H0, g.lo, g.hi, sp["eps"], sp["mu"])
        rn = oinv.invariants(Eo, Ho, g.lo, g.hi, sp["eps"], sp["mu"])
        sc = inv_scales(r0, sp["eps"], sp["mu"])
        assert [r["step"] for r in mix[i][2]] == list(range(2 * steps + 1))
        assert inv_diff(mix[i][2][-1], rn, sc) < tol
