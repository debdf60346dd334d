"""Discrete invariants of Sec. 4, evaluated in physical space. FP64, numpy.

Test infrastructure only (see ``oracle/__init__.py``).

Everything here follows the definitions written in the theorems, not the
spectral shortcuts the CUDA path takes:

* D_w is the N_w x N_w spectral differentiation matrix of Sec. 2.2,
  (D_w)_{jl} = (nu_w/2) (-1)^{j+l} cot(nu_w (w_j - w_l)/2) for j != l, 0 on
  the diagonal, applied along axis w ("D_1 = I (x) I (x) D_x", ...).
* D is the block curl of eq. (maxreformFD).
* Time derivatives come from eq. (hamFD) / Remark 4.2:
  dH/dt = -(1/mu) D E, dE/dt = (1/eps) D H.
* <u, v>_N = (1/N_S) sum_j u_j v_j (Sec. 3; on a cuboid the normalising
  count is N_x N_y N_z).
"""
from __future__ import annotations

import numpy as np


def cot_matrix(n, lo, hi):
    """(D_w)_{jl} = (nu/2)(-1)^{j+l} cot(nu (w_j - w_l)/2), zero diagonal (Sec. 2.2)."""
    nu = 2.0 * np.pi / (hi - lo)
    h = (hi - lo) / n
    j = np.arange(n)
    diff = j[:, None] - j[None, :]
    D = np.zeros((n, n))
    off = diff != 0
    sign = np.where(diff % 2 == 0, 1.0, -1.0)
    D[off] = 0.5 * nu * sign[off] / np.tan(nu * diff[off] * h / 2.0)
    return D


class Operators:
    """D_1, D_2, D_3 and the curl D of a grid, applied to [..][Nz][Ny][Nx] arrays."""

    def __init__(self, nxyz, lo, hi):
        self.n = tuple(nxyz)
        self.Dx = cot_matrix(nxyz[0], lo[0], hi[0])
        self.Dy = cot_matrix(nxyz[1], lo[1], hi[1])
        self.Dz = cot_matrix(nxyz[2], lo[2], hi[2])
        self.ns = nxyz[0] * nxyz[1] * nxyz[2]

    def d(self, w, u):
        """D_{w+1} u: derivative along axis w (0 = x, 1 = y, 2 = z) of a scalar field."""
        if w == 0:
            return np.einsum("jl,...l->...j", self.Dx, u)
        if w == 1:
            return np.einsum("jl,...lx->...jx", self.Dy, u)
        return np.einsum("jl,...lyx->...jyx", self.Dz, u)

    def curl(self, U):
        """D U for U = (U_x, U_y, U_z): the block matrix of eq. (maxreformFD).

        Row 1: -D_3 U_y + D_2 U_z;  row 2: D_3 U_x - D_1 U_z;  row 3: -D_2 U_x + D_1 U_y.
        """
        return np.stack([
            -self.d(2, U[1]) + self.d(1, U[2]),
            self.d(2, U[0]) - self.d(0, U[2]),
            -self.d(1, U[0]) + self.d(0, U[1]),
        ])

    def inner(self, u, v):
        """<u, v>_N = (1/N_S) sum u v, summed over every leading axis too."""
        return float(np.sum(u * v)) / self.ns


def invariants(E, H, lo, hi, eps, mu, ops=None):
    """All discrete invariants of Thm 4.1, 4.3, 4.4 and the divergences of Thm 4.6.

    Returns a dict with
      E1, E2                         scalars
      E3, E4, E5, E6                 arrays of 3 (k = 1, 2, 3, i.e. x, y, z)
      H1, H2                         scalars (Thm 4.3 labels both "H_1"; the
                                     second uses time derivatives and is H_2)
      M1, M2                         arrays of 3
      divE, divH                     discrete L2 norms ||D~.(eps E)||_N,
                                     ||D~.(mu H)||_N (Thm 4.6; the paper's
                                     "Re(D)" does not name a norm)
      divE_max, divH_max             the same fields' max norms
    """
    E = np.asarray(E, np.float64)
    H = np.asarray(H, np.float64)
    nz, ny, nx = E.shape[1:]
    if ops is None:
        ops = Operators((nx, ny, nz), lo, hi)
    inn = ops.inner
    DE = ops.curl(E)
    DH = ops.curl(H)
    Hd = -DE / mu  # dH/dt
    Ed = DH / eps  # dE/dt
    out = {}
    out["E1"] = 0.5 * mu * inn(H, H) + 0.5 * eps * inn(E, E)
    out["E2"] = 0.5 * mu * inn(Hd, Hd) + 0.5 * eps * inn(Ed, Ed)
    E3, E4, E5, E6, M1, M2 = (np.zeros(3) for _ in range(6))
    for k in range(3):
        dkH = np.stack([ops.d(k, H[w]) for w in range(3)])
        dkE = np.stack([ops.d(k, E[w]) for w in range(3)])
        dkHd = np.stack([ops.d(k, Hd[w]) for w in range(3)])
        dkEd = np.stack([ops.d(k, Ed[w]) for w in range(3)])
        E3[k] = 0.5 * mu * inn(dkH, dkH) + 0.5 * eps * inn(dkE, dkE)
        E4[k] = 0.5 * mu * inn(dkHd, dkHd) + 0.5 * eps * inn(dkEd, dkEd)
        E5[k] = 0.5 * mu * inn(H, dkH) + 0.5 * eps * inn(E, dkE)
        E6[k] = 0.5 * mu * inn(Hd, dkHd) + 0.5 * eps * inn(Ed, dkEd)
        M1[k] = inn(H, dkE)  # <H, B_k E>_N
        M2[k] = inn(E, dkH)  # <E, B_k H>_N
    out.update(E3=E3, E4=E4, E5=E5, E6=E6, M1=M1, M2=M2)
    out["H1"] = inn(H, DH) / (2 * eps) + inn(E, DE) / (2 * mu)
    DHd = ops.curl(Hd)
    DEd = ops.curl(Ed)
    out["H2"] = inn(Hd, DHd) / (2 * eps) + inn(Ed, DEd) / (2 * mu)
    divE = eps * (ops.d(0, E[0]) + ops.d(1, E[1]) + ops.d(2, E[2]))
    divH = mu * (ops.d(0, H[0]) + ops.d(1, H[1]) + ops.d(2, H[2]))
    out["divE"] = np.sqrt(inn(divE, divE))
    out["divH"] = np.sqrt(inn(divH, divH))
    out["divE_max"] = float(np.abs(divE).max())
    out["divH_max"] = float(np.abs(divH).max())
    return out
