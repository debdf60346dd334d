"""FP32 precision form against the FP64 oracle at full size (256^3, h = 0.02,
500 steps, random divergence-free fields with sigma = 16) and the literal
FP32 form beside it.  Target: relative L2 error per field <= 1e-5.

The oracle computes the 500-step result as one step of size 500 h (Def. 2.3
with t_end = 500 h), which equals the repeated step to round-off by the group
property pinned in tests/test_oracle_pins.py.
"""
import numpy as np
import pytest

from oracle import scheme
from tests.gpu_util import solver_mod

pytestmark = pytest.mark.gpu

N, H, STEPS, SIGMA = 256, 0.02, 500, 16.0


@pytest.fixture(scope="module")
def case():
    import torch

    mx = solver_mod()
    n = (N, N, N)
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    gen = mx.Solver(n, lo, hi, 1.0, 1.0, mx.MX_FP64, mx.MX_FORM_SPECTRAL)
    gen.load_random(3, SIGMA)
    E0 = torch.empty((3, N, N, N), dtype=torch.float64, device="cuda")
    H0 = torch.empty_like(E0)
    gen.read(E0, H0)
    gen.sync()
    gen.close()
    E0n, H0n = E0.cpu().numpy(), H0.cpu().numpy()
    Eo, Ho = scheme.solve(E0n, H0n, lo, hi, 1.0, 1.0, STEPS * H)
    return E0, H0, Eo, Ho, n, lo, hi


def _field_errors(E, H, Eo, Ho):
    def rel(a, b):
        return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))

    return [rel(E[c], Eo[c]) for c in range(3)] + [rel(H[c], Ho[c]) for c in range(3)]


@pytest.mark.parametrize("form", ["spectral", "literal"])
def test_fp32_error_vs_fp64_oracle_256(case, form):
    import torch

    mx = solver_mod()
    E0, H0, Eo, Ho, n, lo, hi = case
    F = mx.MX_FORM_SPECTRAL if form == "spectral" else mx.MX_FORM_LITERAL
    s = mx.Solver(n, lo, hi, 1.0, 1.0, mx.MX_FP32, F)
    Ef, Hf = E0.float().contiguous(), H0.float().contiguous()
    s.load(Ef, Hf)
    s.step(H, STEPS, 50)
    s.read(Ef, Hf)
    s.sync()
    inv = s.invariants()
    s.close()
    En, Hn = Ef.double().cpu().numpy(), Hf.double().cpu().numpy()
    errs = _field_errors(En, Hn, Eo, Ho)
    print(form, "per-field rel L2", ["%.2e" % e for e in errs])
    e1 = [r["E1"] for r in inv]
    print(form, "E1 rel drift", (max(e1) - min(e1)) / e1[0])
    assert max(errs) <= 1e-5
    # the FP32 path's invariant sums (FP32 per thread or warp, compensated, FP64 across warps and
    # blocks) against the same sums in FP64 over the FP32 state it returned: E1 = (mu <H,H> + eps <E,E>)/2
    e1_fp64 = 0.5 * (np.sum(Hn ** 2) + np.sum(En ** 2)) / float(np.prod(n))
    acc = abs(inv[-1]["E1"] - e1_fp64) / e1_fp64
    print(form, "E1 of the final state: FP32-path sums vs FP64 sums, rel", acc)
    assert acc < 1e-6


def test_fp64_spectral_256_matches_oracle(case):
    mx = solver_mod()
    E0, H0, Eo, Ho, n, lo, hi = case
    s = mx.Solver(n, lo, hi, 1.0, 1.0, mx.MX_FP64, mx.MX_FORM_SPECTRAL)
    Ed, Hd = E0.clone(), H0.clone()
    s.load(Ed, Hd)
    s.step(H, STEPS, 100)
    s.read(Ed, Hd)
    s.sync()
    s.close()
    errs = _field_errors(Ed.cpu().numpy(), Hd.cpu().numpy(), Eo, Ho)
    assert max(errs) <= 1e-12
