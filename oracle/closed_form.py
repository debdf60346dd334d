"""Exact solutions of the continuous Maxwell system used as pins. FP64, numpy.

Test infrastructure only (see ``oracle/__init__.py``).

The scheme is exact in space for fields whose Fourier content lies strictly
inside the Nyquist band (|m_w| < N_w/2): the spectral derivative of such a
field is its true derivative, and the time integration is the exact
exponential.  On those fields the scheme must reproduce these solutions at
the collocation points to round-off (Sec. 5, Tables 4 and 8).
"""
from __future__ import annotations

import numpy as np


def plane_wave_sum(x, y, z, t, params):
    """E, H of sum_j a_j cos(k_j.x + phi_j - omega_j t), H_j = (k_j x a_j)/(mu omega_j) cos(.).

    x, y, z: coordinate arrays of any common shape.  Returns (E, H) with a
    leading component axis of length 3.  Each term solves eq. (maxsys): with
    a_j . k_j = 0 and omega_j^2 = |k_j|^2/(eps mu),
    dH/dt = -(1/mu) curl E and dE/dt = (1/eps) curl H.
    """
    x = np.asarray(x, np.float64)
    E = np.zeros((3,) + x.shape)
    H = np.zeros((3,) + x.shape)
    mu = params["mu"]
    for kj, aj, pj, wj in zip(params["k"], params["a"], params["phi"], params["omega"]):
        ph = np.cos(kj[0] * x + kj[1] * y + kj[2] * z + pj - wj * t)
        bj = np.cross(kj, aj) / (mu * wj)
        for c in range(3):
            E[c] += aj[c] * ph
            H[c] += bj[c] * ph
    return E, H


def plane_wave_energy(params):
    """E1 of a plane-wave sum with distinct +-m_j on a grid that resolves every wave.

    The grid mean of cos^2 is 1/2 and cross terms of distinct resolved waves
    average to 0, so E1 = sum_j (eps |a_j|^2 + mu |b_j|^2)/4 with
    b_j = k_j x a_j / (mu omega_j).
    """
    eps, mu = params["eps"], params["mu"]
    tot = 0.0
    for kj, aj, wj in zip(params["k"], params["a"], params["omega"]):
        bj = np.cross(kj, aj) / (mu * wj)
        tot += 0.25 * (eps * aj @ aj + mu * bj @ bj)
    return tot


def standing_wave(x, y, z, t, kvec=(1, 2, -3), eps=1.0, mu=1.0):
    """Eq. (standing) of Sec. 5.1: the standing wave on [0,2]^3 (needs k_x + k_y + k_z = 0).

    E_x = (k_y - k_z)/(eps sqrt(mu) w) cos(w pi t) cos(k_x pi x) sin(k_y pi y) sin(k_z pi z),
    H_x = sin(w pi t) sin(k_x pi x) cos(k_y pi y) cos(k_z pi z), and cyclically;
    w = sqrt((k_x^2 + k_y^2 + k_z^2)/(eps mu)).
    """
    kx, ky, kz = kvec
    w = np.sqrt((kx * kx + ky * ky + kz * kz) / (eps * mu))
    p = np.pi
    ct, st = np.cos(w * p * t), np.sin(w * p * t)
    amp = 1.0 / (eps * np.sqrt(mu) * w)
    cx, sx = np.cos(kx * p * x), np.sin(kx * p * x)
    cy, sy = np.cos(ky * p * y), np.sin(ky * p * y)
    cz, sz = np.cos(kz * p * z), np.sin(kz * p * z)
    E = np.stack([
        (ky - kz) * amp * ct * cx * sy * sz,
        (kz - kx) * amp * ct * sx * cy * sz,
        (kx - ky) * amp * ct * sx * sy * cz,
    ])
    H = np.stack([st * sx * cy * cz, st * cx * sy * cz, st * cx * cy * sz])
    return E, H


def travelling_wave(x, y, z, t):
    """Sec. 5.2 travelling wave on [0,1]^3, eps = mu = 1:
    E_x = cos(2 pi (x+y+z) - 2 sqrt(3) pi t), E_y = -2 E_x, E_z = E_x,
    H_x = sqrt(3) E_x, H_y = 0, H_z = -sqrt(3) E_x.
    """
    ex = np.cos(2 * np.pi * (x + y + z) - 2 * np.sqrt(3) * np.pi * t)
    E = np.stack([ex, -2 * ex, ex])
    H = np.stack([np.sqrt(3) * ex, np.zeros_like(ex), -np.sqrt(3) * ex])
    return E, H
