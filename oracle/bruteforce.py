"""Brute-force exact flow of the semi-discrete system, tiny grids only. FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The semi-discrete system eq. (maxreformFD) is
    d/dt (sqrt(mu) H, sqrt(eps) E) = (1/sqrt(mu eps)) [[0, -D], [D, 0]] (sqrt(mu) H, sqrt(eps) E)
with D the 3 N_S x 3 N_S block curl built from the cot matrices D_w.
D is real symmetric (D_w antisymmetric), so D = Q diag(lam) Q^T and, as in
Prop. 2.1 (whose proof carries over verbatim from Lambda to D), the flow is
    [[cos(t D / sqrt(mu eps)), -sin(t D / sqrt(mu eps))],
     [sin(t D / sqrt(mu eps)),  cos(t D / sqrt(mu eps))]].
No FFT is used here: this is independent of ``scheme``.
"""
from __future__ import annotations

import numpy as np

from .invariants import cot_matrix


def curl_matrix(nxyz, lo, hi):
    """Dense D of eq. (maxreformFD), acting on (U_x, U_y, U_z) stacked, x-fastest vectors."""
    nx, ny, nz = nxyz
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    D1 = np.kron(Iz, np.kron(Iy, cot_matrix(nx, lo[0], hi[0])))
    D2 = np.kron(Iz, np.kron(cot_matrix(ny, lo[1], hi[1]), Ix))
    D3 = np.kron(cot_matrix(nz, lo[2], hi[2]), np.kron(Iy, Ix))
    Z = np.zeros_like(D1)
    return np.block([[Z, -D3, D2], [D3, Z, -D1], [-D2, D1, Z]])


def exact_flow(E0, H0, lo, hi, eps, mu, t):
    """(E(t), H(t)) of the semi-discrete system by eigendecomposition of D."""
    E0 = np.asarray(E0, np.float64)
    H0 = np.asarray(H0, np.float64)
    nz, ny, nx = E0.shape[1:]
    D = curl_matrix((nx, ny, nz), lo, hi)
    lam, Q = np.linalg.eigh(D)
    arg = t * lam / np.sqrt(mu * eps)
    C = (Q * np.cos(arg)) @ Q.T
    S = (Q * np.sin(arg)) @ Q.T
    u = np.sqrt(mu) * H0.reshape(-1)
    v = np.sqrt(eps) * E0.reshape(-1)
    un = C @ u - S @ v
    vn = S @ u + C @ v
    H = (un / np.sqrt(mu)).reshape(H0.shape)
    E = (vn / np.sqrt(eps)).reshape(E0.shape)
    return E, H
