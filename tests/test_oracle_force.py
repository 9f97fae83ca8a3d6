"""Pins of the fermion-force oracle (no GPU): the force is checked against central finite
differences of the action S = phi^dagger A^-1 phi computed by dense LAPACK solves, so that a wrong
sign, factor, phase or index anywhere in it fails; plus Hermiticity, tracelessness and gauge
covariance."""
import numpy as np
import pytest

from oracle import force as F
from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I


def _herm_direction(rng):
    a = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    h = 0.5 * (a + a.conj().T)
    return h - np.trace(h) / 3 * np.eye(3)


def _expi(h, eps):
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * eps * w)) @ v.conj().T


def _solve_xy(U, phi, dims, mass):
    even = np.nonzero(S.parity(dims) == 0)[0]
    A = F.even_normal_dense(U, dims, mass)
    x = np.zeros_like(phi)
    x[even] = np.linalg.solve(A, phi[even].reshape(-1)).reshape(-1, 3)
    y = S.dslash_parity(U, x, dims, 1)
    return x, y


def _fd_check(dims, links, seed=1, mass=0.3, eps=1e-4):
    """Largest |finite difference - tr(H G)| over the links, relative to the largest |tr(H G)|."""
    rng = np.random.default_rng(seed)
    U = I.make_links(dims, kind="haar", seed=seed)
    phi = I.make_source(dims, seed=seed + 1)
    x, y = _solve_xy(U, phi, dims, mass)
    G = F.fermion_force(U, x, y, dims)
    errs, scale = [], []
    for n, mu in links:
        h = _herm_direction(rng)
        Up, Um = U.copy(), U.copy()
        Up[n, mu] = _expi(h, eps) @ U[n, mu]
        Um[n, mu] = _expi(h, -eps) @ U[n, mu]
        fd = (F.pseudofermion_action_dense(Up, phi, dims, mass) - F.pseudofermion_action_dense(Um, phi, dims, mass)) / (2 * eps)
        want = np.trace(h @ G[n, mu])
        assert abs(want.imag) <= 1e-12 * max(1.0, abs(want.real))
        errs.append(abs(fd - want.real))
        scale.append(abs(want.real))
    return max(errs) / max(scale)


def test_force_matches_finite_differences_every_link_2x2x2x2():
    dims = (2, 2, 2, 2)
    links = [(n, mu) for n in range(S.volume(dims)) for mu in range(4)]
    assert _fd_check(dims, links) <= 1e-6


def test_force_matches_finite_differences_2x4x2x4():
    dims = (2, 4, 2, 4)
    V = S.volume(dims)
    rng = np.random.default_rng(5)
    last_t = [n for n in range(V) if S.coords(dims)[n, 3] == dims[3] - 1]
    links = [(int(n), int(mu)) for n, mu in zip(rng.choice(V, 12, replace=False), rng.integers(0, 4, 12))]
    links += [(last_t[0], 3), (last_t[1], 3)]  # antiperiodic boundary links, both parities
    assert _fd_check(dims, links, seed=3, mass=0.2) <= 1e-6


def test_force_is_traceless_hermitian_and_site_form_agrees():
    dims = (2, 4, 6, 8)
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=2)
    y = I.make_source(dims, seed=3)
    G = F.fermion_force(U, x, y, dims)
    assert np.max(np.abs(G - np.conj(np.swapaxes(G, -1, -2)))) <= 1e-14
    assert np.max(np.abs(np.trace(G, axis1=-2, axis2=-1))) <= 1e-14
    V = S.volume(dims)
    sites = np.arange(V).repeat(4)
    mus = np.tile(np.arange(4), V)
    assert np.max(np.abs(F.fermion_force_links(U, x, y, dims, sites, mus) - G.reshape(-1, 3, 3))) <= 1e-15


def test_force_gauge_covariance():
    """G[U^g, g x, g y](n) = g(n) G[U, x, y](n) g(n)^dagger."""
    dims = (4, 2, 4, 6)
    U = I.make_links(dims, kind="haar", seed=1)
    g = I.make_gauge_transform(dims, seed=4)
    x = I.make_source(dims, seed=2)
    y = I.make_source(dims, seed=3)
    iup, _ = S.neighbour_tables(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[iup[:, mu]], -1, -2))
    gx = np.einsum("sab,sb->sa", g, x)
    gy = np.einsum("sab,sb->sa", g, y)
    lhs = F.fermion_force(Ug, gx, gy, dims)
    rhs = np.einsum("sab,smbc,sdc->smad", g, F.fermion_force(U, x, y, dims), np.conj(g))
    assert np.max(np.abs(lhs - rhs)) <= 1e-13


def test_force_free_field_zero_for_zero_solution():
    dims = (2, 2, 2, 4)
    U = I.make_links(dims, kind="haar", seed=1)
    z = np.zeros((S.volume(dims), 3), np.complex128)
    assert not np.any(F.fermion_force(U, z, I.make_source(dims, seed=2), dims))


@pytest.mark.parametrize("mistake", ["periodic_t", "no_dagger", "eta_shift"])
def test_planted_mistake_in_force_fails_the_finite_difference_pin(monkeypatch, mistake):
    """Plant a plausible mistake in the force only (the action is untouched): the pin must catch it."""
    if mistake == "periodic_t":
        monkeypatch.setattr(F, "_coeff", lambda dims, mu, tbc: 0.5 * S.eta(dims, mu))
    elif mistake == "eta_shift":
        monkeypatch.setattr(F, "_coeff", lambda dims, mu, tbc: 0.5 * S.eta(dims, min(mu + 1, 3)) * S.zeta(dims, mu, tbc))
    else:
        def odd_w(c, U, y, x_fwd):
            yx = np.einsum("sa,sb->sab", y, np.conj(x_fwd))
            return c[:, None, None] * np.einsum("sab,sbc->sac", yx, U)
        monkeypatch.setattr(F, "_odd_w", odd_w)
    dims = (2, 2, 2, 2)
    links = [(n, mu) for n in range(S.volume(dims)) for mu in range(4)]
    assert _fd_check(dims, links) > 1e-3
