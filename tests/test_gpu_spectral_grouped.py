"""The spectral-resident form's grouped-row pass (`k_spectral_grp`): chunks of the rows (±m_y, ±m_z)
that share each |k|² coefficient entry, in segments of 128 columns.  It runs for FP32 table
coefficients when Mx is a multiple of 128 and N_y, N_z are even.  These grids have short y and z
axes, so most row groups are degenerate (m = 0 and the Nyquist index, where -m is m).  Mx = 256
takes two segments per row.

Against the FP64 oracle's literal stepping per field (FP32 1e-5; Alg. 2 with t_end = t_n, which
the group property makes equal to n steps of h, Def. 2.3) and its physical-space invariants.
"""
import numpy as np
import pytest

import synth
from oracle import invariants as oinv
from oracle import scheme
from tests.gpu_util import inv_diff, inv_scales, max_field_rel_l2, run_gpu, solver_mod

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi
GRIDS = [
    ((256, 12, 10), (TWO_PI, 2 * TWO_PI, TWO_PI)),
    ((256, 6, 4), (TWO_PI, TWO_PI, TWO_PI)),
    ((512, 8, 6), (TWO_PI, TWO_PI, 2 * TWO_PI)),
]


@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_grouped_spectral_pass_matches_oracle(gi, device):
    mx = solver_mod()
    n, hi = GRIDS[gi]
    g = synth.Grid(n, (0.0, 0.0, 0.0), hi)
    rng = np.random.default_rng(60 + gi)
    # white noise, not divergence-free: every mode and both polarisations of k x U
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, h, steps = 1.7, 0.6, 0.043, 5
    E, H, inv = run_gpu(g, E0, H0, eps, mu, mx.MX_FP32, mx.MX_FORM_SPECTRAL, h, steps, every=1, device=device)
    Eo, Ho = scheme.step(E0, H0, g.lo, g.hi, eps, mu, h, steps)
    assert max_field_rel_l2(E, H, Eo, Ho) < 1e-5
    assert len(inv) == steps + 1
    r0 = oinv.invariants(E0, H0, g.lo, g.hi, eps, mu)
    rn = oinv.invariants(Eo, Ho, g.lo, g.hi, eps, mu)
    sc = inv_scales(r0, eps, mu)
    assert inv_diff(inv[0], r0, sc) < 1e-5
    assert inv_diff(inv[-1], rn, sc) < 1e-5
