"""Pins of the Wilson-fermion oracle (no GPU): gamma algebra, free-field closed forms,
gamma_5-hermiticity, gauge covariance, dense solves, site-local form."""
import itertools

import numpy as np
import pytest

from oracle import staggered as S
from oracle import wilson as W
from paper_1311_2719_gb300 import inputs as I

LATTICES = [(4, 4, 4, 4), (2, 4, 6, 8)]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _spinor(dims, seed):
    return I.make_spinor(dims, seed)


def test_gamma_algebra():
    g = W.GAMMA
    for mu, nu in itertools.product(range(4), range(4)):
        anti = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)                  # Hermitian
        assert np.allclose(W.GAMMA5 @ g[mu] + g[mu] @ W.GAMMA5, 0)  # gamma5 anticommutes
    assert np.allclose(W.GAMMA5, np.diag([1, 1, -1, -1]))           # DeGrand-Rossi: gamma5 diagonal
    # (1 -+ gamma_mu)/2 are rank-2 projectors (what a spin-projected kernel relies on)
    for mu in range(4):
        for s in (+1, -1):
            P = 0.5 * (np.eye(4) + s * g[mu])
            assert np.allclose(P @ P, P) and np.linalg.matrix_rank(P) == 2


def _cos_sin(dims, k):
    p = [2 * np.pi * k[mu] / dims[mu] for mu in range(4)]
    p[3] += np.pi / dims[3]
    return np.cos(p), np.sin(p)


@pytest.mark.parametrize("dims", LATTICES)
def test_free_field_plane_waves(dims):
    """U = 1: M e^{ipn} psi0 = [1 - 2 kappa sum cos p + 2i kappa sum gamma_mu sin p] e^{ipn} psi0."""
    U = I.make_links(dims, kind="unit")
    kappa = 0.125
    rng = np.random.default_rng(0)
    for k in [(0, 0, 0, 0), (1, 0, 0, 1), (1, 2, 3, 0), (0, 1, 2, dims[3] - 1)]:
        psi0 = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = I.plane_wave(dims, k, [1.0, 0.0, 0.0])[:, 0]
        psi = phase[:, None, None] * psi0[None]
        c, s = _cos_sin(dims, k)
        Mp = (1 - 2 * kappa * c.sum()) * np.eye(4) + 2j * kappa * sum(W.GAMMA[mu] * s[mu] for mu in range(4))
        want = phase[:, None, None] * (Mp @ psi0)[None]
        assert _rel(W.apply_m(U, psi, dims, kappa), want) <= 1e-13
        lam = (1 - 2 * kappa * c.sum()) ** 2 + 4 * kappa * kappa * (s * s).sum()
        MdM = W.apply_mdag(U, W.apply_m(U, psi, dims, kappa), dims, kappa)
        assert _rel(MdM, lam * psi) <= 1e-13


@pytest.mark.parametrize("dims", LATTICES)
def test_gamma5_hermiticity(dims):
    """gamma5 D_W gamma5 = D_W^dagger on Haar links: <y, D x> = <gamma5 D gamma5 y, x>."""
    U = I.make_links(dims, kind="haar", seed=1)
    x, y = _spinor(dims, 3), _spinor(dims, 4)
    lhs = np.vdot(y, W.dslash_w(U, x, dims))
    rhs = np.vdot(W.gamma5(W.dslash_w(U, W.gamma5(y), dims)), x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


@pytest.mark.parametrize("dims", LATTICES)
def test_gauge_covariance(dims):
    U = I.make_links(dims, kind="haar", seed=1)
    G = I.make_gauge_transform(dims, seed=5)
    x = _spinor(dims, 6)
    iup, _ = S.neighbour_tables(dims)
    UG = np.empty_like(U)
    for mu in range(4):
        UG[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(G[iup[:, mu]], -1, -2))
    gx = np.einsum("iab,isb->isa", G, x)
    lhs = W.dslash_w(UG, gx, dims)
    rhs = np.einsum("iab,isb->isa", G, W.dslash_w(U, x, dims))
    assert _rel(lhs, rhs) <= 1e-13


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 4)])
def test_cgnr_matches_dense_solve(dims):
    U = I.make_links(dims, kind="haar", seed=1)
    b = _spinor(dims, 2)
    kappa = 0.12
    n = S.volume(dims) * 12
    cols = []
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        cols.append(W.apply_m(U, e.reshape(-1, 4, 3), dims, kappa).reshape(-1))
    M = np.stack(cols, axis=1)
    G5 = np.kron(np.eye(S.volume(dims)), np.kron(W.GAMMA5, np.eye(3)))
    assert np.max(np.abs(G5 @ M @ G5 - M.conj().T)) <= 1e-14     # gamma5-hermiticity of the matrix
    x_dense = np.linalg.solve(M, b.reshape(-1)).reshape(-1, 4, 3)
    res = W.cgnr(U, b, dims, kappa, tol=1e-13, max_iter=5000)
    assert res["converged"] and res["rel_residual"] <= 1e-11
    assert _rel(res["x"], x_dense) <= 1e-10


def test_site_local_form_matches_full():
    dims = (2, 4, 6, 8)
    U = I.make_links(dims, kind="haar", seed=1)
    x = _spinor(dims, 3)
    sites = np.arange(S.volume(dims))
    assert _rel(W.dslash_w_sites(U, x, dims, sites), W.dslash_w(U, x, dims)) <= 1e-15


@pytest.mark.parametrize("mistake", ["periodic_t", "axes_swapped"])
def test_planted_mistake_in_wilson_oracle_fails_a_pin(monkeypatch, mistake):
    """Plant a plausible mistake in the oracle (on the CPU): some pin must catch it."""
    if mistake == "periodic_t":
        monkeypatch.setattr(S, "zeta", lambda dims, mu, tbc=-1.0: np.ones(S.volume(dims)))
    else:
        monkeypatch.setattr(S, "_axis", lambda mu: [3, 2, 0, 1][mu])
    failed = False
    for pin in (lambda: test_free_field_plane_waves((2, 4, 6, 8)), lambda: test_gauge_covariance((2, 4, 6, 8))):
        try:
            pin()
        except AssertionError:
            failed = True
    assert failed


# ---------------------------------------------------------------- residual checkers (exact values)
#
# x = (1 - eps) M^-1 b (dense LAPACK) leaves b - M x = eps b and M^dagger b - M^dagger M x =
# eps M^dagger b: both relative residuals equal eps exactly, for any eps.


def _wilson_residual_pins(dims):
    U = I.make_links(dims, kind="haar", seed=1)
    b = _spinor(dims, 2)
    kappa = 0.12
    n = S.volume(dims) * 12
    cols = []
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        cols.append(W.apply_m(U, e.reshape(-1, 4, 3), dims, kappa).reshape(-1))
    x_exact = np.linalg.solve(np.stack(cols, axis=1), b.reshape(-1)).reshape(-1, 4, 3)
    for eps in (0.3, 1e-4, 1e-8):
        r = W.residuals(U, (1.0 - eps) * x_exact, b, dims, kappa)
        assert abs(r["rel_residual"] - eps) <= 1e-13, (eps, r)
        assert abs(r["normal_rel_residual"] - eps) <= 1e-13, (eps, r)


def test_wilson_residual_checkers_are_exact():
    _wilson_residual_pins((2, 2, 2, 2))


@pytest.mark.parametrize("mistake", ["no_sqrt", "unnormalised", "normal_wrong_norm"])
def test_planted_wilson_residual_mistake_fails_its_pin(monkeypatch, mistake):
    orig = W.residuals

    def wrong(U, x, b, dims, kappa, tbc=-1.0):
        r = orig(U, x, b, dims, kappa, tbc)
        if mistake == "no_sqrt":
            r = {k: v * v for k, v in r.items()}
        elif mistake == "unnormalised":
            r["rel_residual"] *= float(np.linalg.norm(b))
        else:
            # the normal residual normalised by |b| instead of |M^dagger b|
            rhs = W.apply_mdag(U, b, dims, kappa, tbc)
            nres = rhs - W.apply_mdag(U, W.apply_m(U, x, dims, kappa, tbc), dims, kappa, tbc)
            r["normal_rel_residual"] = float(np.linalg.norm(nres) / np.linalg.norm(b))
        return r

    monkeypatch.setattr(W, "residuals", wrong)
    with pytest.raises(AssertionError):
        _wilson_residual_pins((2, 2, 2, 2))
