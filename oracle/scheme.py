"""Alg. 1 and Alg. 2 of the paper (Sec. 2.4-2.5), FP64, numpy.

Test infrastructure only (see ``oracle/__init__.py``).

Arrays are laid out [component][Nz][Ny][Nx] (x fastest), which is the
paper's vector ordering of Sec. 2.2.  The 3D DFT of the paper,
F_{N_z} (x) F_{N_y} (x) F_{N_x} with entries exp(-2 pi i j k / N) and the
inverse carrying 1/N per axis (Sec. 2.3), is the oracle's own mixed-radix
FFT (``oracle/fft.py``) over the three spatial axes; ``tests/test_oracle_pins.py``
checks it against the DFT matrix and a naive O(N_S^2) 3D DFT written from the
definition.
"""
from __future__ import annotations

import numpy as np

from .fft import fft3, ifft3


def wavenumber_vector(n, lo, hi):
    """a_w of Alg. 2 step 1: (2 pi/(w_R - w_L)) * (0, 1, ..., N/2-1, 0, -N/2+1, ..., -1).

    The Nyquist entry is 0 as in the definition of Omega_w (Sec. 2.3); the
    algorithm listing prints "N_w/2+1" after it, which we read as -N_w/2+1
    (a sign typo: the diagonal of Omega_w fixes it).
    """
    nu = 2.0 * np.pi / (hi - lo)
    m = np.concatenate([np.arange(0, n // 2), [0], np.arange(-n // 2 + 1, 0)]).astype(np.float64)
    return nu * m


def b_vectors(nxyz, lo, hi):
    """b_x, b_y, b_z of Alg. 2 step 2 as arrays of shape [Nz][Ny][Nx].

    b_x = 1_{Nz} (x) 1_{Ny} (x) a_x, b_y = 1 (x) a_y (x) 1, b_z = a_z (x) 1 (x) 1.
    """
    nx, ny, nz = nxyz
    ax = wavenumber_vector(nx, lo[0], hi[0])
    ay = wavenumber_vector(ny, lo[1], hi[1])
    az = wavenumber_vector(nz, lo[2], hi[2])
    bx = np.broadcast_to(ax[None, None, :], (nz, ny, nx)).copy()
    by = np.broadcast_to(ay[None, :, None], (nz, ny, nx)).copy()
    bz = np.broadcast_to(az[:, None, None], (nz, ny, nx)).copy()
    return bx, by, bz


def forward3(u):
    """Alg. 1 step 4 / eq. (tran0): (F_{Nz} (x) F_{Ny} (x) F_{Nx}) u for each component."""
    return fft3(u)


def inverse3(uh):
    """Alg. 2 step 5 / eq. (tran1): (F^{-1}_{Nz} (x) F^{-1}_{Ny} (x) F^{-1}_{Nx}) uh."""
    return ifft3(uh)


def coefficients(nxyz, lo, hi, eps, mu, t):
    """Alg. 2 steps 2-3: Psi, r1, r2 and c11, c12, c13, c22, c23, c33, s12, s13, s23.

    kappa = t / sqrt(mu eps), Psi = kappa^2 (b_x^2 + b_y^2 + b_z^2).
    r1 = (cosh(sqrt(-Psi)) - 1) ./ Psi, r2 = sinh(sqrt(-Psi)) ./ sqrt(-Psi).
    Psi >= 0, so sqrt(-Psi) = i sqrt(Psi), cosh(i s) = cos s and
    sinh(i s)/(i s) = sin s / s.  Where Psi = 0 (k = 0, or t = 0) the two
    quotients are 0/0; we take their limits r1 = -1/2, r2 = 1, which makes
    the update the identity there, as the exponential of a zero matrix is.
    """
    bx, by, bz = b_vectors(nxyz, lo, hi)
    kappa = t / np.sqrt(mu * eps)
    psi = kappa * kappa * (bx * bx + by * by + bz * bz)
    s = np.sqrt(psi)
    zero = psi == 0.0
    safe_psi = np.where(zero, 1.0, psi)
    safe_s = np.where(zero, 1.0, s)
    r1 = np.where(zero, -0.5, (np.cos(s) - 1.0) / safe_psi)
    r2 = np.where(zero, 1.0, np.sin(s) / safe_s)
    k2 = kappa * kappa
    c = {
        "c11": 1.0 + k2 * (bz * bz + by * by) * r1,
        "c12": -k2 * by * bx * r1,
        "s12": 1j * kappa * bz * r2,
        "c22": 1.0 + k2 * (bz * bz + bx * bx) * r1,
        "c13": -k2 * bz * bx * r1,
        "s13": 1j * kappa * by * r2,
        "c33": 1.0 + k2 * (by * by + bx * bx) * r1,
        "c23": -k2 * bz * by * r1,
        "s23": 1j * kappa * bx * r2,
    }
    return c


def update(Hh, Eh, c, eps, mu):
    """Alg. 2 step 4: scale by sqrt(mu), sqrt(eps), apply the 6x6 per-k map, unscale.

    Hh, Eh: complex spectra [3][Nz][Ny][Nx].  Returns the new (Hh, Eh).
    """
    smu, seps = np.sqrt(mu), np.sqrt(eps)
    Hx, Hy, Hz = smu * Hh[0], smu * Hh[1], smu * Hh[2]
    Ex, Ey, Ez = seps * Eh[0], seps * Eh[1], seps * Eh[2]
    c11, c12, c13 = c["c11"], c["c12"], c["c13"]
    c22, c23, c33 = c["c22"], c["c23"], c["c33"]
    s12, s13, s23 = c["s12"], c["s13"], c["s23"]
    nHx = c11 * Hx + c12 * Hy + c13 * Hz + s12 * Ey - s13 * Ez
    nHy = c12 * Hx + c22 * Hy + c23 * Hz - s12 * Ex + s23 * Ez
    nHz = c13 * Hx + c23 * Hy + c33 * Hz + s13 * Ex - s23 * Ey
    nEx = c11 * Ex + c12 * Ey + c13 * Ez - s12 * Hy + s13 * Hz
    nEy = c12 * Ex + c22 * Ey + c23 * Ez + s12 * Hx - s23 * Hz
    nEz = c13 * Ex + c23 * Ey + c33 * Ez - s13 * Hx + s23 * Hy
    Hn = np.stack([nHx, nHy, nHz]) / smu
    En = np.stack([nEx, nEy, nEz]) / seps
    return Hn, En


def solve(E0, H0, lo, hi, eps, mu, t_end, check_imag=True):
    """Def. 2.3 Steps 2-4 with one step of size t_end: Alg. 1 then Alg. 2.

    E0, H0: real fields [3][Nz][Ny][Nx] at the collocation points.
    Returns real (E, H) at t_end.
    """
    E0 = np.asarray(E0, dtype=np.float64)
    H0 = np.asarray(H0, dtype=np.float64)
    nz, ny, nx = E0.shape[1:]
    Eh = forward3(E0)
    Hh = forward3(H0)
    c = coefficients((nx, ny, nz), lo, hi, eps, mu, t_end)
    Hh, Eh = update(Hh, Eh, c, eps, mu)
    E = inverse3(Eh)
    H = inverse3(Hh)
    if check_imag:
        scale = max(np.abs(E).max(), np.abs(H).max(), 1e-300)
        imag = max(np.abs(E.imag).max(), np.abs(H.imag).max())
        assert imag <= 1e-12 * scale, f"imaginary residue {imag:.3e} vs scale {scale:.3e}"
    return E.real.copy(), H.real.copy()


def step(E0, H0, lo, hi, eps, mu, h, nsteps):
    """The scheme repeated: nsteps applications of one step of size h.

    Each application is Alg. 1 + Alg. 2 with t_end = h on the fields the
    previous one returned (the time-stepping reading of Def. 2.3 with
    Delta t = t_end / N_t).
    """
    E, H = np.asarray(E0, np.float64), np.asarray(H0, np.float64)
    for _ in range(int(nsteps)):
        E, H = solve(E, H, lo, hi, eps, mu, h)
    return E, H
