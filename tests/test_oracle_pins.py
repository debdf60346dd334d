"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties one part of ``oracle/`` to the paper's definitions, to a
closed form, to brute force or to a value the paper prints, so that a
plausible slip (a dropped term, a flipped sign, a transposed operand, a
wrong Nyquist convention, a wrong normalisation) fails at least one test.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import bruteforce, closed_form as cf, fft as offt, invariants as inv, scheme

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def dft_matrix(n):
    """(F_N)_{jk} = (exp(2 pi i / N))^{-jk}, written from its definition (Sec. 2.3)."""
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


# ---------------------------------------------------------------- transforms


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12])
def test_forward_is_paper_dft_along_each_axis(n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    F = dft_matrix(n)
    np.testing.assert_allclose(scheme.forward3(u.reshape(1, 1, n)).ravel(), F @ u, atol=1e-12)
    np.testing.assert_allclose(scheme.forward3(u.reshape(1, n, 1)).ravel(), F @ u, atol=1e-12)
    np.testing.assert_allclose(scheme.forward3(u.reshape(n, 1, 1)).ravel(), F @ u, atol=1e-12)
    Finv = np.conj(F) / n  # (F^{-1})_{jk} = (1/N) exp(2 pi i/N)^{jk}
    np.testing.assert_allclose(Finv @ F, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(scheme.inverse3((F @ u).reshape(1, 1, n)).ravel(), u, atol=1e-12)


@pytest.mark.parametrize("n", list(range(1, 41)) + [64, 96, 125, 128, 160, 243, 250])
def test_oracle_fft_is_dft_matrix(n):
    """The oracle's mixed-radix FFT against the transform's matrix, forward and inverse, for every
    length up to 40 (radices 2, 3, 5, their products and the prime lengths finished by the
    definition) and longer 2/3/5-smooth lengths where a wrong twiddle index or digit order shows."""
    rng = np.random.default_rng(1000 + n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    F = dft_matrix(n)
    scale = np.abs(x).max() * n
    np.testing.assert_allclose(offt.fft(x), x @ F.T, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(offt.ifft(x), x @ np.conj(F).T / n, rtol=0, atol=1e-13 * scale / n)
    np.testing.assert_allclose(offt.ifft(offt.fft(x)), x, rtol=0, atol=1e-13 * np.abs(x).max())


def _naive_dft3(u, sign):
    """sum over all N_S points of u_j exp(sign 2 pi i (jx kx/Nx + jy ky/Ny + jz kz/Nz)): the 3D DFT
    written out with one N_S x N_S exponent matrix (no factorisation into axes)."""
    nz, ny, nx = u.shape[-3:]
    jz, jy, jx = (a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"))
    ph = (np.outer(jx, jx) / nx + np.outer(jy, jy) / ny + np.outer(jz, jz) / nz)
    W = np.exp(sign * 2j * np.pi * ph)
    return (u.reshape(u.shape[:-3] + (-1,)) @ W.T).reshape(u.shape)


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 10, 6), (5, 9, 7)])
def test_oracle_fft3_is_naive_3d_dft(shape):
    """forward3/inverse3 against the naive O(N_S^2) 3D DFT at 8^3 and on cuboids with radices 2, 3, 5
    (and the prime lengths 5, 7 by the definition), [Nz][Ny][Nx] with x fastest."""
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal((2,) + shape)
    X = scheme.forward3(u)
    ref = _naive_dft3(u, -1)
    np.testing.assert_allclose(X, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    ns = int(np.prod(shape))
    np.testing.assert_allclose(scheme.inverse3(X), _naive_dft3(X, +1) / ns, rtol=0, atol=1e-12 * np.abs(u).max())
    # Parseval: sum |u|^2 = (1/N_S) sum |X|^2
    assert abs(np.sum(np.abs(X) ** 2) / ns - np.sum(u ** 2)) < 1e-12 * np.sum(u ** 2)


def test_oracle_fft3_agrees_with_library_fft_at_size():
    """At sizes where a naive DFT is out of reach, the library transform (numpy.fft) serves as a pin
    of the oracle's own: 30 x 32 x 48 and a 512-long line."""
    rng = np.random.default_rng(5)
    u = rng.standard_normal((48, 32, 30))
    ref = np.fft.fftn(u)
    np.testing.assert_allclose(scheme.forward3(u), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    x = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    np.testing.assert_allclose(offt.fft(x), np.fft.fft(x), rtol=0, atol=1e-12 * np.abs(x).sum())


def test_forward_is_kronecker_product_in_x_fastest_order():
    nx, ny, nz = 6, 4, 2
    rng = np.random.default_rng(7)
    u = rng.standard_normal((nz, ny, nx))
    K = np.kron(dft_matrix(nz), np.kron(dft_matrix(ny), dft_matrix(nx)))
    np.testing.assert_allclose(scheme.forward3(u).reshape(-1), K @ u.reshape(-1), atol=1e-11)


@pytest.mark.parametrize("n,L", [(2, 2 * np.pi), (4, 2 * np.pi), (6, 3.0), (8, 2.0), (16, 5.5)])
def test_cot_matrix_is_spectral_derivative_with_nyquist_zero(n, L):
    """D_w (cot formula) = F^{-1} diag(i a_w) F with a_w's Nyquist entry 0."""
    D = inv.cot_matrix(n, 0.0, L)
    F = dft_matrix(n)
    a = scheme.wavenumber_vector(n, 0.0, L)
    assert a[n // 2] == 0.0
    spectral = (np.conj(F) / n) @ np.diag(1j * a) @ F
    np.testing.assert_allclose(D, spectral.real, atol=1e-12 * max(1.0, np.abs(D).max()))
    assert np.abs(spectral.imag).max() < 1e-12 * max(1.0, np.abs(D).max())
    # D is antisymmetric; a Nyquist-only field is static under it.
    np.testing.assert_allclose(D, -D.T, atol=1e-13 * max(1.0, np.abs(D).max()))
    x = np.arange(n) * L / n
    np.testing.assert_allclose(D @ np.cos(np.pi * n / L * x), 0.0, atol=1e-12 * max(1, np.abs(D).max()))
    if n >= 4:  # a resolved mode differentiates exactly
        nu = 2 * np.pi / L
        np.testing.assert_allclose(D @ np.sin(nu * x), nu * np.cos(nu * x), atol=1e-12 * n)


# ------------------------------------------------------ scheme vs brute force


@pytest.mark.parametrize(
    "n,hi,eps,mu,t",
    [
        ((4, 4, 4), (2 * np.pi,) * 3, 1.0, 1.0, 0.37),
        ((4, 6, 8), (1.0, 2.0, 3.0), 1.7, 0.6, 0.37),
        ((4, 6, 8), (1.0, 2.0, 3.0), 1.7, 0.6, -3.1),
        ((6, 4, 2), (2.0, 1.0, 1.5), 0.3, 2.5, 11.0),
        ((2, 4, 4), (1.0, 1.0, 1.0), 1.0, 1.0, 0.9),
    ],
)
def test_scheme_matches_bruteforce_exponential(n, hi, eps, mu, t):
    """Alg. 1 + Alg. 2 equals the exact flow of eq. (maxreformFD) built without FFTs."""
    g = synth.Grid(n, (0.0, 0.0, 0.0), hi)
    rng = np.random.default_rng(sum(n))
    E0 = rng.standard_normal((3,) + g.shape)  # not divergence free: tests every block
    H0 = rng.standard_normal((3,) + g.shape)
    Eb, Hb = bruteforce.exact_flow(E0, H0, g.lo, g.hi, eps, mu, t)
    Es, Hs = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, t)
    np.testing.assert_allclose(Es, Eb, atol=1e-12 * 10)
    np.testing.assert_allclose(Hs, Hb, atol=1e-12 * 10)


def test_bruteforce_small_time_is_the_ode():
    """(u(dt) - u(-dt)) / (2 dt) ~ the right-hand side of eq. (maxreformFD)."""
    g = synth.Grid((4, 4, 6), (0, 0, 0), (1.0, 1.3, 2.0))
    rng = np.random.default_rng(3)
    E0, H0 = rng.standard_normal((3,) + g.shape), rng.standard_normal((3,) + g.shape)
    eps, mu, dt = 1.3, 0.7, 1e-5
    Ep, Hp = bruteforce.exact_flow(E0, H0, g.lo, g.hi, eps, mu, dt)
    Em, Hm = bruteforce.exact_flow(E0, H0, g.lo, g.hi, eps, mu, -dt)
    ops = inv.Operators(g.n, g.lo, g.hi)
    np.testing.assert_allclose((Hp - Hm) / (2 * dt), -ops.curl(E0) / mu, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose((Ep - Em) / (2 * dt), ops.curl(H0) / eps, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------- closed forms


def _errors(E, H, Ee, He, npts):
    l2 = np.sqrt((np.sum((E - Ee) ** 2) + np.sum((H - He) ** 2)) / npts)
    linf = max(np.abs(E - Ee).max(), np.abs(H - He).max())
    return l2, linf


@pytest.mark.parametrize("N", [8, 16])
def test_standing_wave_example1(N):
    """Sec. 5.1: one step of size t_end reproduces eq. (standing); errors no larger than Table 'error s2'."""
    gold = json.load(open(GOLDEN))["example1_solution_errors"]
    g = synth.Grid((N, N, N), (0, 0, 0), (2, 2, 2))
    E0, H0 = synth.standing_wave_fields(g)
    x, y, z = g.mesh()
    for i, t in enumerate(gold["t_end"]):
        E, H = scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, float(t))
        Ee, He = cf.standing_wave(x, y, z, float(t))
        l2, linf = _errors(E, H, Ee, He, g.npoints)
        assert l2 <= max(gold[f"N{N}"]["L2"][i], 1e-13)
        assert linf <= max(gold[f"N{N}"]["Linf"][i], 1e-13)


@pytest.mark.parametrize("N", [8, 16])
def test_travelling_wave_example2(N):
    """Sec. 5.2: the travelling wave; errors no larger than Table 'error s'."""
    gold = json.load(open(GOLDEN))["example2_solution_errors"]
    g = synth.Grid((N, N, N), (0, 0, 0), (1, 1, 1))
    E0, H0 = synth.travelling_wave_fields(g)
    x, y, z = g.mesh()
    for i, t in enumerate(gold["t_end"]):
        E, H = scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, float(t))
        Ee, He = cf.travelling_wave(x, y, z, float(t))
        l2, linf = _errors(E, H, Ee, He, g.npoints)
        assert l2 <= max(gold[f"N{N}"]["L2"][i], 1e-13)
        assert linf <= max(gold[f"N{N}"]["Linf"][i], 1e-13)


def test_closed_forms_solve_maxwell():
    """The closed forms themselves: finite differences in t against curls taken by hand."""
    x, y, z = np.meshgrid(*(np.linspace(0.1, 1.7, 5),) * 3, indexing="ij")
    p = synth.plane_wave_params(5, eps=2.0, mu=0.5)
    dt = 1e-6
    for fn in (lambda t: cf.plane_wave_sum(x, y, z, t, p), lambda t: cf.standing_wave(x, y, z, t),
               lambda t: cf.travelling_wave(x, y, z, t)):
        E1, H1 = fn(0.3 + dt)
        E0, H0 = fn(0.3 - dt)
        Ec, Hc = fn(0.3)
        assert np.abs(E1 - E0).max() > 1e-9  # not static
    # plane-wave sum: dE/dt = (1/eps) curl H, checked per wave analytically
    for kj, aj, wj in zip(p["k"], p["a"], p["omega"]):
        assert abs(kj @ aj) < 1e-12
        np.testing.assert_allclose(wj ** 2, kj @ kj / (p["eps"] * p["mu"]))
    # standing wave: the (1,2,-3) vector sums to zero, which makes it a solution
    kx, ky, kz = 1, 2, -3
    assert kx + ky + kz == 0


@pytest.mark.parametrize("seed", [1, 2])
def test_plane_wave_sum_many_steps(seed):
    """Config-1 style input on a cuboid with eps != mu: 100 steps of h equal the closed form."""
    g = synth.Grid((16, 12, 10), (0, 0, 0), (2 * np.pi, 2 * np.pi, 2 * np.pi))
    p = synth.plane_wave_params(seed, eps=2.0, mu=0.5, kmax=3)
    E0, H0 = synth.plane_wave_fields(g, p)
    x, y, z = g.mesh()
    Ec0, Hc0 = cf.plane_wave_sum(x, y, z, 0.0, p)
    np.testing.assert_allclose(E0, Ec0, atol=1e-13)
    np.testing.assert_allclose(H0, Hc0, atol=1e-13)
    E, H = scheme.step(E0, H0, g.lo, g.hi, 2.0, 0.5, 0.01, 100)
    Ee, He = cf.plane_wave_sum(x, y, z, 1.0, p)
    assert np.abs(E - Ee).max() < 1e-12
    assert np.abs(H - He).max() < 1e-12


# --------------------------------------------------------- group properties


def test_group_property_and_reversibility():
    g = synth.Grid((8, 6, 10), (0, 0, 0), (1.0, 2.0, 1.5))
    E0, H0 = synth.random_divfree_fields(g, seed=11, sigma=4.0)
    eps, mu = 1.5, 0.8
    En, Hn = scheme.step(E0, H0, g.lo, g.hi, eps, mu, 0.05, 40)
    E1, H1 = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, 2.0)
    np.testing.assert_allclose(En, E1, atol=1e-12)
    np.testing.assert_allclose(Hn, H1, atol=1e-12)
    Eb, Hb = scheme.step(En, Hn, g.lo, g.hi, eps, mu, -0.05, 40)
    np.testing.assert_allclose(Eb, E0, atol=1e-12)
    np.testing.assert_allclose(Hb, H0, atol=1e-12)


# -------------------------------------------------------------- invariants


def test_invariants_on_hand_computed_fields():
    """Beltrami field H = (0, sin x, cos x) (curl H = H) and E = (0, cos x, -sin x), on [0,2 pi]^3.

    By hand: <H,H>_N = <E,E>_N = 1; D H = H, D E = E; d_x H = -E... so
    E1 = (mu + eps)/2, H1 = 1/(2 eps) + 1/(2 mu), M1_x = <H, d_x E> = -1, M2_x = +1,
    E3 = ((mu + eps)/2, 0, 0), and both divergences vanish.
    """
    g = synth.Grid((8, 6, 4))
    x, y, z = g.mesh()
    zero = np.zeros_like(x)
    H = np.stack([zero, np.sin(x), np.cos(x)])
    E = np.stack([zero, np.cos(x), -np.sin(x)])
    eps, mu = 1.7, 0.4
    r = inv.invariants(E, H, g.lo, g.hi, eps, mu)
    np.testing.assert_allclose(r["E1"], (mu + eps) / 2, rtol=1e-13)
    np.testing.assert_allclose(r["H1"], 1 / (2 * eps) + 1 / (2 * mu), rtol=1e-13)
    np.testing.assert_allclose(r["M1"], [-1, 0, 0], atol=1e-13)
    np.testing.assert_allclose(r["M2"], [1, 0, 0], atol=1e-13)
    np.testing.assert_allclose(r["E3"], [(mu + eps) / 2, 0, 0], atol=1e-13)
    # dH/dt = -(1/mu) D E = -E/mu, dE/dt = (1/eps) D H = H/eps
    np.testing.assert_allclose(r["E2"], 0.5 * mu / mu ** 2 + 0.5 * eps / eps ** 2, rtol=1e-13)
    np.testing.assert_allclose(r["H2"], (1 / (2 * eps)) / mu ** 2 + (1 / (2 * mu)) / eps ** 2, rtol=1e-13)
    np.testing.assert_allclose(r["E4"], [r["E2"], 0, 0], atol=1e-13)
    assert r["divE"] < 1e-13 and r["divH"] < 1e-13


def test_divergence_of_a_gradient_field():
    """E = (sin x, 0, 0): D~.(eps E) = eps cos x, so ||.||_N = eps/sqrt(2), max = eps."""
    g = synth.Grid((8, 4, 4))
    x, y, z = g.mesh()
    E = np.stack([np.sin(x), 0 * x, 0 * x])
    H = np.stack([0 * x, 0 * x, np.sin(2 * y)])
    r = inv.invariants(E, H, g.lo, g.hi, 3.0, 0.5)
    np.testing.assert_allclose(r["divE"], 3.0 / np.sqrt(2), rtol=1e-13)
    np.testing.assert_allclose(r["divE_max"], 3.0, rtol=1e-13)
    assert r["divH"] < 1e-13


def test_energy_of_plane_wave_sums_and_standing_wave():
    g = synth.Grid((12, 10, 8))
    p = synth.plane_wave_params(4, eps=1.3, mu=2.1, kmax=3)
    E, H = synth.plane_wave_fields(g, p)
    r = inv.invariants(E, H, g.lo, g.hi, 1.3, 2.1)
    np.testing.assert_allclose(r["E1"], cf.plane_wave_energy(p), rtol=1e-13)
    # linearly polarised waves carry no helicity
    assert abs(r["H1"]) < 1e-12
    # Sec. 5.1 at t = 0: amplitudes (5, -4, -1)/sqrt(14), mean of each product 1/8:
    # E1 = (1/2) * (25 + 16 + 1)/14 / 8 = 3/16
    gs = synth.Grid((8, 8, 8), (0, 0, 0), (2, 2, 2))
    Es, Hs = synth.standing_wave_fields(gs)
    rs = inv.invariants(Es, Hs, gs.lo, gs.hi, 1.0, 1.0)
    np.testing.assert_allclose(rs["E1"], 3.0 / 16.0, rtol=1e-13)


def _scale(r, eps, mu):
    """Cauchy-Schwarz bounds used to normalise drifts of invariants that can be ~0."""
    e1, e2 = abs(r["E1"]), abs(r["E2"])
    return {
        "E1": e1, "E2": e2, "E3": np.abs(r["E3"]).sum(), "E4": np.abs(r["E4"]).sum(),
        "H1": np.sqrt(e1 * e2) / np.sqrt(eps * mu) + 1e-300,
        "H2": np.sqrt(e2 * np.abs(r["E4"]).sum()) / np.sqrt(eps * mu) + 1e-300,
        "M1": 2 * np.sqrt(e1 * np.abs(r["E3"]).sum()) / np.sqrt(eps * mu),
    }


def test_invariants_conserved_by_scheme():
    """Thm 4.1, 4.3, 4.4, 4.6: conserved to round-off; E5 = E6 = 0; M2 = -M1."""
    g = synth.Grid((10, 8, 12), (0, 0, 0), (2.0, 1.0, 3.0))
    E0, H0 = synth.random_divfree_fields(g, seed=5, sigma=5.0)
    # add a gradient part so the divergence is non-zero and must be conserved too
    x, y, z = g.mesh()
    E0 = E0 + 0.3 * np.stack([np.cos(np.pi * x), 0 * x, 0 * x])
    eps, mu = 2.0, 0.7
    r0 = inv.invariants(E0, H0, g.lo, g.hi, eps, mu)
    sc = _scale(r0, eps, mu)
    for t in (0.3, 7.0, 150.0):
        E, H = scheme.solve(E0, H0, g.lo, g.hi, eps, mu, t)
        r = inv.invariants(E, H, g.lo, g.hi, eps, mu)
        for key in ("E1", "E2", "E3", "E4", "H1", "H2", "M1"):
            drift = np.abs(np.asarray(r[key]) - np.asarray(r0[key])).max() / sc[key]
            assert drift < 1e-13, (key, t, drift)
        np.testing.assert_allclose(r["M2"], -r["M1"], atol=1e-13 * sc["M1"])
        assert np.abs(r["E5"]).max() < 1e-14 * sc["E1"] * 10
        assert np.abs(r["E6"]).max() < 1e-14 * sc["E2"] * 10
        np.testing.assert_allclose(r["divE"], r0["divE"], rtol=1e-12)
        assert r0["divE"] > 0.1
        assert r["divH"] < 1e-12 * np.sqrt(sc["E3"])
    # the random fields are not trivially invariant-free
    assert abs(r0["H1"]) > 1e-3 * sc["H1"] and np.abs(r0["M1"]).max() > 1e-3 * sc["M1"]


def test_paper_energy_and_divergence_tables():
    """Tables 'error e2', 'error e', 'error D2', 'error D': our drifts are no larger."""
    gold = json.load(open(GOLDEN))
    for N in (8, 16):
        g = synth.Grid((N, N, N), (0, 0, 0), (2, 2, 2))
        E0, H0 = synth.standing_wave_fields(g)
        r0 = inv.invariants(E0, H0, g.lo, g.hi, 1.0, 1.0)
        for t in (1.0, 20.0):
            E, H = scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, t)
            r = inv.invariants(E, H, g.lo, g.hi, 1.0, 1.0)
            for key in ("E1", "E2"):
                rel = abs(r[key] - r0[key]) / abs(r0[key])
                assert rel <= max(gold["example1_energy_drift"]["max_relative_drift_E1_to_E4"], 2e-15)
            assert r["divE_max"] <= max(gold["divergence"]["max_abs"], 1e-13)
            assert r["divH_max"] <= max(gold["divergence"]["max_abs"], 1e-13)


# ------------------------------------------------------- symplecticity, convergence


def _omega(E_a, H_a, E_b, H_b, eps, mu):
    """Symplectic form of Thm 4.5 in the scaled variables u = sqrt(mu) H, v = sqrt(eps) E:
    omega(a, b) = <v_a, u_b> - <u_a, v_b> (sum over all points and components)."""
    ua, va = np.sqrt(mu) * H_a, np.sqrt(eps) * E_a
    ub, vb = np.sqrt(mu) * H_b, np.sqrt(eps) * E_b
    return float(np.sum(va * ub) - np.sum(ua * vb))


def test_symplecticity_thm45():
    """The step preserves dE ^ dH: omega(R a, R b) = omega(a, b) for two independent states."""
    g = synth.Grid((8, 10, 6), (0, 0, 0), (1.0, 1.4, 0.9))
    rng = np.random.default_rng(45)
    Ea, Ha, Eb, Hb = (rng.standard_normal((3,) + g.shape) for _ in range(4))
    eps, mu = 1.6, 0.7
    w0 = _omega(Ea, Ha, Eb, Hb, eps, mu)
    for t in (0.3, 4.0):
        Ea1, Ha1 = scheme.solve(Ea, Ha, g.lo, g.hi, eps, mu, t)
        Eb1, Hb1 = scheme.solve(Eb, Hb, g.lo, g.hi, eps, mu, t)
        w1 = _omega(Ea1, Ha1, Eb1, Hb1, eps, mu)
        assert abs(w1 - w0) < 1e-12 * (np.abs(Ea).sum() + np.abs(Eb).sum())
    # and it is not trivially zero
    assert abs(w0) > 1.0


def test_spectral_convergence_thm34():
    """Thm 3.4: for smooth, non-band-limited data the error decays faster than any power of N.

    Initial fields E = curl A with A = (0, 0, exp(sin x) exp(cos y) cos z) (smooth, divergence
    free, all wavenumbers present), H = 0; reference: the same scheme on a 48^3 grid, compared
    at the coarse collocation points (which the fine grid contains since 48 is a multiple).
    """
    def fields(n):
        g = synth.Grid((n, n, n))
        x, y, z = g.mesh()
        a = np.exp(np.sin(x)) * np.exp(np.cos(y))
        # curl (0, 0, A_z) = (d_y A_z, -d_x A_z, 0)
        Ex = a * (-np.sin(y)) * np.cos(z)
        Ey = -(a * np.cos(x)) * np.cos(z)
        E = np.stack([Ex, Ey, 0 * x])
        return g, E, 0 * E

    t = 0.7
    gF, EF, HF = fields(48)
    EfT, HfT = scheme.solve(EF, HF, gF.lo, gF.hi, 1.0, 1.0, t)
    errs = []
    for n in (8, 12, 16, 24):
        g, E, H = fields(n)
        Et, Ht = scheme.solve(E, H, g.lo, g.hi, 1.0, 1.0, t)
        s = 48 // n
        ref_E = EfT[:, ::s, ::s, ::s]
        ref_H = HfT[:, ::s, ::s, ::s]
        errs.append(np.sqrt(np.mean((Et - ref_E) ** 2) + np.mean((Ht - ref_H) ** 2)))
    # faster than algebraic: each refinement gains more than the previous power law predicts
    assert errs[-1] < 1e-6 * errs[0]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(n2 / n1) for i, (n1, n2) in enumerate([(8, 12), (12, 16), (16, 24)])]
    assert rates[-1] > rates[0] > 2.0
