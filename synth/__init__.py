"""Seeded synthetic inputs for the periodic 3D Maxwell solver.

This module only draws and lays out input data.  It holds none of the
scheme's arithmetic: no exponential update, no invariants.  Both the CPU
oracle (``oracle/``) and the CUDA path receive the arrays made here.

Layout of every field array: ``[3][Nz][Ny][Nx]`` (component, then z, y, x
with x fastest), the vector ordering of the paper's Sec. 2.2 (index
``Nx*Ny*(l-1) + Nx*(k-1) + j``).  Component order is (x, y, z).

Two input families follow the paper's workloads:

* ``plane_wave_params`` / ``plane_wave_fields``: a sum of divergence-free
  plane waves ``E = sum_j a_j cos(k_j.x + phi_j)`` and
  ``H = sum_j (k_j x a_j)/(mu*omega_j) cos(k_j.x + phi_j)``, with integer
  wave vectors, the closed-form family of Sec. 5 (standing and travelling
  waves) generalised to several waves.
* ``random_divfree_fields``: Gaussian white noise, Fourier transformed,
  multiplied by ``exp(-|k|^2 / (2 sigma^2))``, projected perpendicular to k,
  Nyquist planes and k = 0 zeroed, transformed back.  Real and divergence
  free on the grid.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Grid",
    "plane_wave_params",
    "plane_wave_fields",
    "random_divfree_fields",
    "standing_wave_fields",
    "travelling_wave_fields",
]


class Grid:
    """Collocation grid of Def. 2.3 Step 1: even N_w, spacing (w_R - w_L)/N_w."""

    def __init__(self, n, lo=(0.0, 0.0, 0.0), hi=(2 * np.pi, 2 * np.pi, 2 * np.pi)):
        self.n = tuple(int(v) for v in n)  # (Nx, Ny, Nz)
        self.lo = tuple(float(v) for v in lo)
        self.hi = tuple(float(v) for v in hi)
        for v in self.n:
            if v < 2 or v % 2:
                raise ValueError("grid sizes must be even and >= 2")

    @property
    def shape(self):
        """Array shape [Nz][Ny][Nx] of one field component."""
        return (self.n[2], self.n[1], self.n[0])

    @property
    def npoints(self):
        return self.n[0] * self.n[1] * self.n[2]

    def axis(self, w):
        """Collocation points x_j = x_L + (j-1) h along axis w (0=x, 1=y, 2=z)."""
        n = self.n[w]
        h = (self.hi[w] - self.lo[w]) / n
        return self.lo[w] + h * np.arange(n)

    def mesh(self):
        """Coordinate arrays X, Y, Z of shape [Nz][Ny][Nx]."""
        z, y, x = np.meshgrid(self.axis(2), self.axis(1), self.axis(0), indexing="ij")
        return x, y, z

    def nu(self):
        return tuple(2 * np.pi / (self.hi[w] - self.lo[w]) for w in range(3))


def plane_wave_params(seed, nwaves=4, kmax=3, eps=1.0, mu=1.0, nu=(1.0, 1.0, 1.0)):
    """Draw ``nwaves`` plane waves with integer index vectors m_j, |m_ji| <= kmax.

    Wave vector k_j = (nu_x m_x, nu_y m_y, nu_z m_z).  No two waves share +-m,
    so their energies add.  Amplitudes a_j are Gaussian, projected
    perpendicular to k_j; phases are uniform on [0, 2 pi).
    Returns a dict with arrays m (n,3), k (n,3), a (n,3), phi (n,), omega (n,)
    and the scalars eps, mu.
    """
    rng = np.random.default_rng(seed)
    ms = []
    while len(ms) < nwaves:
        m = rng.integers(-kmax, kmax + 1, size=3)
        if not m.any():
            continue
        if any((m == q).all() or (m == -q).all() for q in ms):
            continue
        ms.append(m)
    m = np.array(ms, dtype=np.int64)
    k = m * np.asarray(nu, dtype=np.float64)[None, :]
    a = rng.standard_normal((nwaves, 3))
    khat = k / np.linalg.norm(k, axis=1, keepdims=True)
    a = a - (a * khat).sum(axis=1, keepdims=True) * khat
    phi = rng.uniform(0.0, 2 * np.pi, size=nwaves)
    omega = np.linalg.norm(k, axis=1) / np.sqrt(eps * mu)
    return {"m": m, "k": k, "a": a, "phi": phi, "omega": omega, "eps": float(eps), "mu": float(mu)}


def plane_wave_fields(grid: Grid, params, dtype=np.float64):
    """Evaluate the initial fields of a plane-wave sum on the grid (time 0).

    Returns (E, H), each of shape [3][Nz][Ny][Nx].
    """
    x, y, z = grid.mesh()
    E = np.zeros((3,) + grid.shape)
    H = np.zeros((3,) + grid.shape)
    mu = params["mu"]
    for kj, aj, pj, wj in zip(params["k"], params["a"], params["phi"], params["omega"]):
        ph = np.cos(kj[0] * x + kj[1] * y + kj[2] * z + pj)
        bj = np.cross(kj, aj) / (mu * wj)
        for c in range(3):
            E[c] += aj[c] * ph
            H[c] += bj[c] * ph
    return E.astype(dtype), H.astype(dtype)


def standing_wave_fields(grid: Grid, kvec=(1, 2, -3), eps=1.0, mu=1.0, dtype=np.float64):
    """Initial values of the standing wave of Sec. 5.1 (time 0) on [0,2]^3.

    E_x ~ (k_y - k_z) cos(k_x pi x) sin(k_y pi y) sin(k_z pi z) / (eps sqrt(mu) w),
    and cyclic; H = 0 at t = 0 because it carries sin(w pi t).
    """
    kx, ky, kz = kvec
    w = np.sqrt((kx * kx + ky * ky + kz * kz) / (eps * mu))
    x, y, z = grid.mesh()
    amp = 1.0 / (eps * np.sqrt(mu) * w)
    E = np.stack([
        (ky - kz) * amp * np.cos(kx * np.pi * x) * np.sin(ky * np.pi * y) * np.sin(kz * np.pi * z),
        (kz - kx) * amp * np.sin(kx * np.pi * x) * np.cos(ky * np.pi * y) * np.sin(kz * np.pi * z),
        (kx - ky) * amp * np.sin(kx * np.pi * x) * np.sin(ky * np.pi * y) * np.cos(kz * np.pi * z),
    ])
    H = np.zeros_like(E)
    return E.astype(dtype), H.astype(dtype)


def travelling_wave_fields(grid: Grid, dtype=np.float64):
    """Initial values of the travelling wave of Sec. 5.2 (time 0) on [0,1]^3, eps = mu = 1.

    E_x = cos(2 pi (x+y+z)), E_y = -2 E_x, E_z = E_x, H_x = sqrt(3) E_x, H_y = 0,
    H_z = -sqrt(3) E_x.
    """
    x, y, z = grid.mesh()
    ex = np.cos(2 * np.pi * (x + y + z))
    E = np.stack([ex, -2 * ex, ex])
    H = np.stack([np.sqrt(3) * ex, np.zeros_like(ex), -np.sqrt(3) * ex])
    return E.astype(dtype), H.astype(dtype)


def random_divfree_fields(grid: Grid, seed, sigma=8.0, rms=1.0, dtype=np.float64):
    """Random real divergence-free E and H (independent), smooth spectrum.

    White noise -> FFT -> * exp(-|k|^2/(2 sigma^2)) -> project perpendicular
    to k -> Nyquist planes and k = 0 zeroed -> inverse FFT -> scaled so that
    each field has the given RMS per component.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid.n
    nu = grid.nu()
    mx = np.fft.rfftfreq(nx, d=1.0 / nx)
    my = np.fft.fftfreq(ny, d=1.0 / ny)
    mz = np.fft.fftfreq(nz, d=1.0 / nz)
    KZ, KY, KX = np.meshgrid(nu[2] * mz, nu[1] * my, nu[0] * mx, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    nyq = np.zeros_like(k2, dtype=bool)
    nyq[:, :, nx // 2] = True
    nyq[:, ny // 2, :] = True
    nyq[nz // 2, :, :] = True
    env = np.exp(-k2 / (2.0 * sigma * sigma))
    env[nyq] = 0.0
    env[0, 0, 0] = 0.0
    safe = np.where(k2 > 0, k2, 1.0)
    out = []
    for _ in range(2):
        noise = rng.standard_normal((3,) + grid.shape)
        spec = np.fft.rfftn(noise, axes=(1, 2, 3)) * env[None]
        kdot = (KX * spec[0] + KY * spec[1] + KZ * spec[2]) / safe
        spec[0] -= kdot * KX
        spec[1] -= kdot * KY
        spec[2] -= kdot * KZ
        f = np.fft.irfftn(spec, s=grid.shape, axes=(1, 2, 3))
        scale = np.sqrt(np.mean(f * f))
        if scale > 0:
            f *= rms / scale
        out.append(f)
    return out[0].astype(dtype), out[1].astype(dtype)
