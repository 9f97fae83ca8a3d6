"""Pins of the CPU oracle against what the physics and the mathematics fix (no GPU).

Each check is independent of the oracle's own code path: closed forms (free-field
momenta, pure-gauge solutions through an FFT), operator identities (anti-hermiticity,
gauge covariance, the even-odd block structure), brute force (dense matrices and a
LAPACK solve on tiny lattices) and fixture invariants (unitarity, det = 1).
"""
import itertools

import numpy as np
import pytest

from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I

LATTICES = [(4, 4, 4, 4), (2, 4, 6, 8)]


def _sin2(dims, k, tbc=-1.0):
    s = 0.0
    for mu in range(4):
        p = 2 * np.pi * k[mu] / dims[mu]
        if mu == 3 and tbc < 0:
            p += np.pi / dims[3]
        s += np.sin(p) ** 2
    return s


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- fixtures


@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_link_fixture_is_su3(kind):
    U = I.make_links((4, 4, 2, 2), kind=kind, seed=1).reshape(-1, 3, 3)
    eye = np.eye(3)
    uu = np.conj(np.swapaxes(U, -1, -2)) @ U
    assert np.max(np.abs(uu - eye)) <= 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) <= 1e-14


def test_haar_fixture_is_not_degenerate():
    # Haar measure: E|U_ab|^2 = 1/3 and E[U_ab] = 0.
    U = I.make_links((8, 8, 8, 8), kind="haar", seed=1).reshape(-1, 3, 3)
    assert abs(np.mean(np.abs(U) ** 2) - 1.0 / 3.0) < 5e-3
    assert abs(np.mean(U)) < 5e-3


def test_reconstruct12_round_trip():
    U = I.make_links((4, 4, 4, 4), kind="haar", seed=7).reshape(-1, 3, 3)
    c = S.reconstruct_third_row(U[:, 0, :], U[:, 1, :])
    assert np.max(np.abs(c - U[:, 2, :])) <= 1e-15 * 10


# ---------------------------------------------------------------- free field (closed form)


@pytest.mark.parametrize("dims", LATTICES)
def test_free_field_d_squared_is_minus_sum_sin2(dims):
    """With U = 1, D^2 = -sum_mu sin^2 p_mu on plane waves (antiperiodic t momenta)."""
    U = I.make_links(dims, kind="unit")
    rng = np.random.default_rng(0)
    ks = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 1), (1, 2, 3, 0), (dims[0] // 2, 1, 1, dims[3] - 1)]
    for k in ks:
        colour = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        w = I.plane_wave(dims, k, colour)
        d2 = S.dslash(U, S.dslash(U, w, dims), dims)
        assert _rel(d2, -_sin2(dims, k) * w) <= 1e-13, k


@pytest.mark.parametrize("dims", LATTICES)
def test_free_field_mdagm_on_even_plane_waves(dims):
    """A = m^2 - D_eo D_oe acting on the even restriction of a plane wave gives (m^2 + sum sin^2) times it."""
    U = I.make_links(dims, kind="unit")
    even = (S.parity(dims) == 0)[:, None]
    m = 0.1
    for k in [(1, 0, 0, 0), (1, 1, 2, 3), (0, 3, 1, 2)]:
        w = np.where(even, I.plane_wave(dims, k, [1.0, 0.5j, -0.25]), 0.0)
        lam = m * m + _sin2(dims, k)
        assert _rel(S.mdagm(U, w, dims, m), lam * w) <= 1e-13


def test_free_field_spectrum_4444():
    """Eigenvalues of the dense free D on 4^4 (antiperiodic t): +-i sqrt(sum sin^2 p), 3 colours each."""
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="unit")
    Dm = S.dense_operator(lambda v: S.dslash(U, v, dims), S.volume(dims))
    ev = np.linalg.eigvals(Dm)
    assert np.max(np.abs(ev.real)) <= 1e-12
    want = []
    for k in itertools.product(*[range(L) for L in dims]):
        want += [_sin2(dims, k)] * 3
    got = np.sort(np.abs(ev) ** 2)
    assert np.max(np.abs(got - np.sort(want))) <= 1e-12
    # The distinct values are 0.5, 1.5, 2.5, 3.5 with 96, 288, 288, 96 eigenvalues.
    vals, counts = np.unique(np.round(got, 9), return_counts=True)
    assert np.allclose(vals, [0.5, 1.5, 2.5, 3.5])
    assert list(counts) == [96, 288, 288, 96]
    # Spectrum symmetric under lambda -> -lambda (staggered chiral symmetry eps D eps = -D).
    assert np.allclose(np.sort(ev.imag), np.sort(-ev.imag), atol=1e-12)


def test_free_field_cg_converges_in_four_iterations():
    """On 4^4 free field A has 4 distinct eigenvalues, so exact CG ends in <= 4 steps (allow 5)."""
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="unit")
    b = I.make_source(dims, seed=2)
    res = S.cg_solve(U, b, dims, mass=0.1, tol=1e-10, max_iter=50)
    assert res["converged"] and res["iterations"] <= 5
    assert res["true_rel_residual"] <= 1e-10


# ---------------------------------------------------------------- operator identities


@pytest.mark.parametrize("dims", LATTICES)
def test_anti_hermiticity(dims):
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=11)
    y = I.make_source(dims, seed=12)
    lhs = np.vdot(y, S.dslash(U, x, dims))
    rhs = np.vdot(S.dslash(U, y, dims), x)
    assert abs(lhs + rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(y)


@pytest.mark.parametrize("dims", LATTICES)
def test_gauge_covariance(dims):
    """D[U^G](G x) = G D[U] x with U^G_mu(n) = G(n) U_mu(n) G(n+mu)^dagger."""
    U = I.make_links(dims, kind="haar", seed=1)
    G = I.make_gauge_transform(dims, seed=5)
    x = I.make_source(dims, seed=3)
    iup, _ = S.neighbour_tables(dims)
    UG = np.empty_like(U)
    for mu in range(4):
        UG[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(G[iup[:, mu]], -1, -2))
    lhs = S.dslash(UG, np.einsum("iab,ib->ia", G, x), dims)
    rhs = np.einsum("iab,ib->ia", G, S.dslash(U, x, dims))
    assert _rel(lhs, rhs) <= 1e-13


@pytest.mark.parametrize("dims", LATTICES)
def test_even_odd_block_structure(dims):
    """D(x_e, 0) = (0, D_oe x_e) and (m^2 - D^2)(x_e, 0) = (A x_e, 0)."""
    U = I.make_links(dims, kind="haar", seed=1)
    par = S.parity(dims)
    x = I.make_source(dims, seed=4)
    xe = np.where((par == 0)[:, None], x, 0.0)
    dx = S.dslash(U, xe, dims)
    assert np.max(np.abs(dx[par == 0])) == 0.0
    assert _rel(S.dslash_parity(U, x, dims, 1), dx) == 0.0
    full = 0.01 * xe - S.dslash(U, dx, dims)
    assert np.max(np.abs(full[par == 1])) == 0.0
    assert _rel(S.mdagm(U, x, dims, 0.1), full) <= 1e-15


def test_neighbour_tables_are_inverse_and_local():
    dims = (2, 4, 6, 8)
    iup, idn = S.neighbour_tables(dims)
    c = S.coords(dims)
    V = S.volume(dims)
    for mu in range(4):
        assert np.array_equal(idn[iup[:, mu], mu], np.arange(V))
        d = (c[iup[:, mu]] - c) % np.array(dims)
        e = np.zeros(4, int)
        e[mu] = 1
        assert np.all(d == e)
    # parity flips along every hop
    par = S.parity(dims)
    assert np.all(par[iup] != par[:, None])


# ---------------------------------------------------------------- brute force solves


@pytest.mark.parametrize("dims,kind", [((2, 2, 2, 2), "haar"), ((2, 4, 6, 8), "haar"), ((2, 2, 2, 2), "near_identity")])
def test_dense_solve_matches_cg(dims, kind):
    """Dense A on the even sites (built column by column) vs CG; A Hermitian with spectrum >= m^2."""
    U = I.make_links(dims, kind=kind, seed=1)
    m = 0.1
    par = S.parity(dims)
    ev_idx = np.nonzero(par == 0)[0]
    V = S.volume(dims)

    def apply_a(v_even):
        full = np.zeros((V, 3), np.complex128)
        full[ev_idx] = v_even
        return S.mdagm(U, full, dims, m)[ev_idx]

    A = S.dense_operator(apply_a, len(ev_idx))
    assert np.max(np.abs(A - np.conj(A.T))) <= 1e-14
    lam = np.linalg.eigvalsh(A)
    assert lam.min() >= m * m * (1 - 1e-12)
    b = I.make_source(dims, seed=2)
    x_dense = np.linalg.solve(A, b[ev_idx].reshape(-1)).reshape(-1, 3)
    res = S.cg_solve(U, b, dims, m, tol=1e-12, max_iter=2000)
    assert res["converged"]
    assert _rel(res["x"][ev_idx], x_dense) <= 1e-10
    assert res["true_rel_residual"] <= 1e-12
    # y = D_oe x on the odd sites
    assert _rel(res["y"], S.dslash_parity(U, res["x"], dims, 1)) <= 1e-15


def test_dense_dslash_anti_hermitian_imaginary_spectrum():
    dims = (2, 4, 6, 8)
    U = I.make_links(dims, kind="haar", seed=1)
    Dm = S.dense_operator(lambda v: S.dslash(U, v, dims), S.volume(dims))
    assert np.max(np.abs(Dm + np.conj(Dm.T))) <= 1e-15
    ev = np.linalg.eigvals(Dm)
    assert np.max(np.abs(ev.real)) <= 1e-12
    assert np.max(np.abs(ev)) <= 4.0 + 1e-12  # |D| <= sum_mu |(T - T^-1)/2| <= 4


def _free_solve_fft(c, dims, m, tbc=-1.0):
    """Closed-form solve of (m^2 - D^2) X = c for U = 1 through a twisted 4-D FFT."""
    L0, L1, L2, L3 = dims
    shp = (L3, L2, L1, L0)
    n3 = np.arange(L3)[:, None, None, None, None]
    twist = np.exp(-1j * np.pi * n3 / L3) if tbc < 0 else np.ones_like(n3)
    f = c.reshape(shp + (3,)) * twist
    F = np.fft.fftn(f, axes=(0, 1, 2, 3))
    k3, k2, k1, k0 = np.meshgrid(*[np.arange(L) for L in shp], indexing="ij")
    p = [2 * np.pi * k0 / L0, 2 * np.pi * k1 / L1, 2 * np.pi * k2 / L2, 2 * np.pi * k3 / L3 + (np.pi / L3 if tbc < 0 else 0)]
    lam = m * m + sum(np.sin(q) ** 2 for q in p)
    X = np.fft.ifftn(F / lam[..., None], axes=(0, 1, 2, 3)) / twist
    return X.reshape(-1, 3)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8)])
def test_pure_gauge_closed_form_solution(dims):
    """U_mu(n) = G(n) G(n+mu)^dagger gives A[U] = G A[1] G^dagger, so x = G FFT-solve(G^dagger b)."""
    G = I.make_gauge_transform(dims, seed=9)
    iup, _ = S.neighbour_tables(dims)
    U = np.empty((S.volume(dims), 4, 3, 3), np.complex128)
    for mu in range(4):
        U[:, mu] = G @ np.conj(np.swapaxes(G[iup[:, mu]], -1, -2))
    m = 0.2
    b = I.make_source(dims, seed=2)
    even = (S.parity(dims) == 0)[:, None]
    be = np.where(even, b, 0.0)
    gdb = np.einsum("iba,ib->ia", np.conj(G), be)      # G^dagger b
    x_closed = np.einsum("iab,ib->ia", G, _free_solve_fft(gdb, dims, m))
    assert np.max(np.abs(x_closed[~even[:, 0]])) <= 1e-12   # stays on the even sites
    res = S.cg_solve(U, b, dims, m, tol=1e-13, max_iter=500)
    assert res["converged"]
    assert _rel(res["x"], x_closed) <= 1e-11


# ---------------------------------------------------------------- planted mistakes fail a pin


def _pins_pass(monkeypatch_ctx=None):
    """A compact subset of the pins; returns False as soon as one fails."""
    dims = (2, 4, 6, 8)
    try:
        test_free_field_d_squared_is_minus_sum_sin2(dims)
        test_anti_hermiticity(dims)
        test_gauge_covariance(dims)
        test_pure_gauge_closed_form_solution(dims)
    except AssertionError:
        return False
    return True


def test_pins_pass_unmodified():
    assert _pins_pass()


@pytest.mark.parametrize("mistake", ["eta_dropped", "periodic_t", "axes_swapped", "eta_shifted"])
def test_planted_mistake_fails_a_pin(monkeypatch, mistake):
    """Plant a plausible mistake in the oracle (on the CPU) and check that some pin catches it."""
    if mistake == "eta_dropped":
        monkeypatch.setattr(S, "eta", lambda dims, mu: np.ones(S.volume(dims)))
    elif mistake == "periodic_t":
        monkeypatch.setattr(S, "zeta", lambda dims, mu, tbc=-1.0: np.ones(S.volume(dims)))
    elif mistake == "axes_swapped":
        monkeypatch.setattr(S, "_axis", lambda mu: [3, 2, 0, 1][mu])
    elif mistake == "eta_shifted":
        orig = S.coords

        def eta_wrong(dims, mu):
            c = orig(dims)
            return np.where(c[:, : mu + 1].sum(axis=1) % 2 == 0, 1.0, -1.0)
        monkeypatch.setattr(S, "eta", eta_wrong)
    assert not _pins_pass()


# ---------------------------------------------------------------- site-local oracle == full oracle


@pytest.mark.parametrize("dims", [(2, 4, 6, 8), (4, 4, 4, 4)])
def test_site_local_forms_match_full_lattice_forms(dims):
    """The sampled-site forms used at large volume agree with the full-lattice definition."""
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=3)
    V = S.volume(dims)
    sites = np.arange(V)
    assert _rel(S.dslash_sites(U, x, dims, sites), S.dslash(U, x, dims)) <= 1e-15
    ev = sites[S.parity(dims) == 0]
    full = S.mdagm(U, x, dims, 0.3)
    assert _rel(S.mdagm_sites(U, x, dims, 0.3, ev[::3]), full[ev[::3]]) <= 1e-14
    iup, idn = S.neighbour_tables(dims)
    a, b = S.neighbour_tables_of_sites(dims, sites)
    assert np.array_equal(a, iup) and np.array_equal(b, idn)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 8)])
def test_full_system_solve_matches_dense(dims):
    """x = M^-1 b for M = m + D on the full lattice: CG on M^dagger M vs LAPACK on the dense M."""
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    m = 0.1
    V = S.volume(dims)
    M = S.dense_operator(lambda v: S.apply_m(U, v, dims, m), V)
    x_dense = np.linalg.solve(M, b.reshape(-1)).reshape(-1, 3)
    res = S.solve_full(U, b, dims, m, tol=1e-13, max_iter=5000)
    assert res["rel_residual"] <= 1e-11
    assert _rel(res["x"], x_dense) <= 1e-10


# ---------------------------------------------------------------- residual checkers (exact values)
#
# Every GPU solve test recomputes the residual of the GPU's solution with the oracle's checkers, so
# the checkers are pinned to exact values: with x_exact from a dense LAPACK solve, the scaled
# x = (1 - eps) x_exact leaves the residual b - A x = eps b, i.e. a relative residual of eps
# exactly, for any eps (up to the O(1e-15) rounding of the dense solve). A missing square root
# (eps^2), a missing or wrong normalisation (eps |b|, eps |b_e| / |b|) or a residual that ignores
# x fails it.

RES_EPS = (0.3, 1e-4, 1e-8)


def _dense_even_solution(U, b, dims, m):
    """x_e = A^-1 b_e by LAPACK on the dense even-site A; full-lattice vector, odd half 0."""
    ev_idx = np.nonzero(S.parity(dims) == 0)[0]
    V = S.volume(dims)

    def apply_a(v_even):
        full = np.zeros((V, 3), np.complex128)
        full[ev_idx] = v_even
        return S.mdagm(U, full, dims, m)[ev_idx]

    A = S.dense_operator(apply_a, len(ev_idx))
    x = np.zeros((V, 3), np.complex128)
    x[ev_idx] = np.linalg.solve(A, b[ev_idx].reshape(-1)).reshape(-1, 3)
    return x


def _dense_full_solution(U, b, dims, m):
    """x = M^-1 b on both parities (M = m + D) by LAPACK on the dense M."""
    M = S.dense_operator(lambda v: S.apply_m(U, v, dims, m), S.volume(dims))
    return np.linalg.solve(M, b.reshape(-1)).reshape(-1, 3)


def _residual_pins(dims):
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)  # odd half non-zero: the even checker must ignore it
    m = 0.5
    xe = _dense_even_solution(U, b, dims, m)
    xf = _dense_full_solution(U, b, dims, m)
    for eps in RES_EPS:
        got = S.true_residual(U, (1.0 - eps) * xe, b, dims, m)
        assert abs(got - eps) <= 1e-13, ("true_residual", eps, got)
        got = S.full_residual(U, (1.0 - eps) * xf, b, dims, m)
        assert abs(got - eps) <= 1e-13, ("full_residual", eps, got)


def _residual_pins_pass():
    try:
        for dims in ((2, 2, 2, 2), (2, 4, 6, 8)):
            _residual_pins(dims)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 8)])
def test_residual_checkers_are_exact_on_scaled_dense_solutions(dims):
    _residual_pins(dims)


@pytest.mark.parametrize("mistake", ["no_sqrt", "unnormalised", "full_b_norm", "ignores_x_sign"])
def test_planted_residual_mistake_fails_its_pin(monkeypatch, mistake):
    """Plant a plausible mistake in the oracle's residual checkers (on the CPU): the exact-value pin
    must catch it."""
    def norm2(a):
        return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)

    def even(dims, v):
        return np.where((S.parity(dims) == 0)[:, None], v, 0.0)

    def wrong_true(U, x, b, dims, mass, tbc=-1.0):
        be = even(dims, b)
        if mistake == "ignores_x_sign":
            res = be + S.mdagm(U, x, dims, mass, tbc)
        else:
            res = be - S.mdagm(U, x, dims, mass, tbc)
        if mistake == "no_sqrt":
            return norm2(res) / norm2(be)
        if mistake == "unnormalised":
            return float(np.sqrt(norm2(res)))
        if mistake == "full_b_norm":
            return float(np.sqrt(norm2(res) / norm2(b)))
        return float(np.sqrt(norm2(res) / norm2(be)))

    monkeypatch.setattr(S, "true_residual", wrong_true)
    assert not _residual_pins_pass()
