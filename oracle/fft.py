"""The oracle's own fast Fourier transform: recursive mixed radix (2, 3, 5). FP64, numpy.

Test infrastructure only (see ``oracle/__init__.py``).

Definition followed (Sec. 2.3 of the paper): the 1D transform of length N is
    X_k = sum_{j=0}^{N-1} x_j exp(-2 pi i j k / N)                       (forward)
    x_j = (1/N) sum_{k=0}^{N-1} X_k exp(+2 pi i j k / N)                 (inverse)
and the 3D transform is F_{Nz} (x) F_{Ny} (x) F_{Nx}: the 1D transform along
each axis of a [..][Nz][Ny][Nx] array.

Algorithm (Cooley-Tukey, decimation in time, one prime factor at a time): for
N = p m with p the smallest of 2, 3, 5 dividing N, split x into the p
subsequences y_r[l] = x_{l p + r} (l = 0..m-1), transform each (length m), then
    X_{k + m q} = sum_{r=0}^{p-1} exp(-2 pi i r q / p) exp(-2 pi i r k / N) Y_r[k]
for k = 0..m-1, q = 0..p-1.  A length with another prime factor is finished by
the transform's definition (its N x N matrix).  Nothing here calls a library
transform; ``numpy.fft`` appears only as a pin in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


def _roots(n, sign):
    """exp(sign 2 pi i j / n) for j = 0..n-1 (the angle reduced exactly: j < n)."""
    return np.exp(sign * 2j * np.pi * np.arange(n) / n)


def _dft_matrix_first(x, sign):
    """The definition: X_k = sum_j exp(sign 2 pi i j k / n) x_j along axis 0."""
    n = x.shape[0]
    j = np.arange(n)
    W = _roots(n, sign)[np.outer(j, j) % n]  # W[k, j]
    return np.tensordot(W, x, axes=([1], [0]))


def _fft_first(x, sign):
    """Unnormalised transform along axis 0 of every line x[:, ...] (sign -1 forward, +1 inverse)."""
    n = x.shape[0]
    if n == 1:
        return x.astype(np.complex128, copy=True)
    p = next((q for q in (2, 3, 5) if n % q == 0), None)
    if p is None:
        return _dft_matrix_first(x.astype(np.complex128), sign)
    m = n // p
    rest = x.shape[1:]
    # y[l, r, ...] = x[l p + r, ...]: the p decimated subsequences, transformed along l
    y = x.reshape((m, p) + rest)
    Y = _fft_first(y, sign)  # Y[k, r, ...] = DFT_m of subsequence r
    # twiddles exp(sign 2 pi i r k / n)
    k = np.arange(m)
    r = np.arange(p)
    tw = _roots(n, sign)[np.outer(k, r) % n].reshape((m, p) + (1,) * len(rest))
    Z = Y * tw
    # the p-point DFT across r: X[q, k, ...] = sum_r exp(sign 2 pi i r q / p) Z[k, r, ...]
    wp = _roots(p, sign)
    X = np.empty((p, m) + rest, np.complex128)
    for q in range(p):
        acc = Z[:, 0].copy()
        for rr in range(1, p):
            acc += wp[(rr * q) % p] * Z[:, rr]
        X[q] = acc
    return X.reshape((n,) + rest)  # index k + m q is row-major (q, k)


def _lines(x, axis, sign):
    """_fft_first over every line along `axis`, taking the lines in groups of a few hundred so
    that a group's intermediate arrays stay in cache (the same arithmetic for every line)."""
    x = np.moveaxis(np.asarray(x), axis, 0)
    n = x.shape[0]
    flat = np.ascontiguousarray(x.reshape(n, -1))
    out = np.empty(flat.shape, np.complex128)
    cols = max(256, (1 << 16) // n)
    for c in range(0, flat.shape[1], cols):
        out[:, c:c + cols] = _fft_first(np.ascontiguousarray(flat[:, c:c + cols]), sign)
    return np.moveaxis(out.reshape(x.shape), 0, axis)


def fft(x, axis=-1):
    """Forward 1D transform (unnormalised, exp(-2 pi i jk/N)) along `axis`."""
    return _lines(x, axis, -1)


def ifft(X, axis=-1):
    """Inverse 1D transform (exp(+2 pi i jk/N) and the factor 1/N) along `axis`."""
    return _lines(X, axis, +1) / np.shape(X)[axis]


def fft3(u):
    """(F_{Nz} (x) F_{Ny} (x) F_{Nx}) u over the last three axes ([..][Nz][Ny][Nx])."""
    out = np.asarray(u)
    for ax in (-1, -2, -3):
        out = fft(out, ax)
    return out


def ifft3(uh):
    """(F^{-1}_{Nz} (x) F^{-1}_{Ny} (x) F^{-1}_{Nx}) uh over the last three axes."""
    out = np.asarray(uh)
    for ax in (-1, -2, -3):
        out = ifft(out, ax)
    return out
