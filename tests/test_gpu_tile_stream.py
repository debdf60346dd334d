"""The access-pattern measurement of the fused z pass (mx_tile_stream): every tile width moves the
spectrum through shared memory and back unchanged, reports a positive rate, and bad arguments are
refused before anything runs."""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import solver_mod

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cols", [4, 8, 16])
@pytest.mark.parametrize("shape", [(64, 32, 512), (48, 6, 96), (16, 2, 2)])
def test_tile_stream_leaves_the_spectrum_unchanged(cols, shape):
    import torch

    mx = solver_mod()
    m, ny, nz = shape
    if m % cols:
        pytest.skip("columns per tile must divide mx")
    rng = np.random.default_rng(5)
    host = rng.standard_normal(6 * nz * ny * m * 2).astype(np.float32)
    buf = torch.tensor(host, device="cuda")
    gbs = mx.tile_stream(buf.data_ptr(), m, ny, nz, cols, reps=2)
    torch.cuda.synchronize()
    assert gbs > 0.0
    assert np.array_equal(buf.cpu().numpy(), host)


def test_tile_stream_rejects_bad_arguments():
    import torch

    mx = solver_mod()
    buf = torch.zeros(6 * 8 * 4 * 8 * 2, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    v = C.c_double(0)
    bad = [(p, 8, 4, 8, 5, 1),            # columns per tile
           (p, 6, 4, 8, 4, 1),            # mx not a multiple of the columns
           (p + 8, 8, 4, 8, 4, 1),        # misaligned
           (p, 8, 4, 600, 4, 1),          # nz above 512
           (p, 8, 4, 8, 4, 0)]            # no timed launch
    for args in bad:
        assert mx.mx_tile_stream(C.c_void_p(args[0]), *args[1:], C.byref(v)) == mx.MX_E_INVAL
    assert mx.mx_tile_stream(None, 8, 4, 8, 4, 1, C.byref(v)) == mx.MX_E_INVAL
