"""Helpers shared by the GPU tests: run the CUDA path through the C ABI."""
import numpy as np

INV_KEYS = ("E1", "E2", "E3", "E4", "H1", "H2", "M1", "M2", "divE", "divH")


def solver_mod():
    from paper_2210_06232_gb300 import maxexp

    return maxexp


def run_gpu(grid, E0, H0, eps, mu, precision, form, h, nsteps, every=1, device=True):
    """Load, step, read through libmaxexp; returns (E, H, invariant records) as float64 numpy."""
    import torch

    mx = solver_mod()
    dt = torch.float64 if precision == mx.MX_FP64 else torch.float32
    s = mx.Solver(grid.n, grid.lo, grid.hi, eps, mu, precision, form)
    try:
        if device:
            Ed = torch.tensor(np.asarray(E0), dtype=dt, device="cuda")
            Hd = torch.tensor(np.asarray(H0), dtype=dt, device="cuda")
            s.load(Ed, Hd)
            if nsteps:
                s.step(h, nsteps, every)
            s.read(Ed, Hd)
            s.sync()
            E, H = Ed.double().cpu().numpy(), Hd.double().cpu().numpy()
        else:
            npdt = np.float64 if precision == mx.MX_FP64 else np.float32
            s.load(np.ascontiguousarray(E0, npdt), np.ascontiguousarray(H0, npdt))
            if nsteps:
                s.step(h, nsteps, every)
            E, H = s.read_numpy()
            E, H = E.astype(np.float64), H.astype(np.float64)
        inv = s.invariants()
    finally:
        s.close()
    return E, H, inv


def rel_l2(E, H, Er, Hr):
    num = np.sqrt(np.sum((E - Er) ** 2) + np.sum((H - Hr) ** 2))
    den = np.sqrt(np.sum(Er ** 2) + np.sum(Hr ** 2))
    return num / max(den, 1e-300)


def field_rel_l2(E, H, Er, Hr):
    """Relative L2 error of each of the six fields (E_x, E_y, E_z, H_x, H_y, H_z) against its reference."""
    out = []
    for X, R in ((E, Er), (H, Hr)):
        for c in range(3):
            den = np.sqrt(np.sum(np.asarray(R[c]) ** 2))
            out.append(float(np.sqrt(np.sum((np.asarray(X[c]) - np.asarray(R[c])) ** 2)) / max(den, 1e-300)))
    return out


def max_field_rel_l2(E, H, Er, Hr):
    """The worst of the six per-field relative L2 errors (the per-field tolerance is on this)."""
    return max(field_rel_l2(E, H, Er, Hr))


def inv_scales(r, eps, mu):
    """Cauchy-Schwarz bounds to normalise invariants that may be ~0."""
    e1, e2 = abs(r["E1"]), abs(r["E2"])
    e3, e4 = float(np.abs(r["E3"]).sum()), float(np.abs(r["E4"]).sum())
    b = np.sqrt(eps * mu)
    return {
        "E1": e1, "E2": e2, "E3": e3, "E4": e4,
        "H1": np.sqrt(e1 * e2) / b + 1e-300, "H2": np.sqrt(e2 * e4) / b + 1e-300,
        "M1": 2 * np.sqrt(e1 * e3) / b + 1e-300, "M2": 2 * np.sqrt(e1 * e3) / b + 1e-300,
        "divE": np.sqrt(6 * eps * e3) + 1e-300, "divH": np.sqrt(6 * mu * e3) + 1e-300,
    }


def inv_diff(a, b, scales):
    """max over keys of |a - b| / scale."""
    worst = 0.0
    for k in INV_KEYS:
        d = np.abs(np.asarray(a[k], float) - np.asarray(b[k], float)).max() / scales[k]
        worst = max(worst, float(d))
    return worst
