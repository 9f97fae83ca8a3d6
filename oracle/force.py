"""Plain FP64 CPU oracle for the staggered fermion force: the derivative of the even-site
pseudofermion action with respect to the gauge links.

TEST INFRASTRUCTURE ONLY: only the test-suite and the benchmark's CPU-baseline leg import it.

The paper's hybrid molecular dynamics program (§2) is the caller of its CG (§4), which returns x on
one parity and "the solution on the second half lattice" y = D_oe x; the paper states no formula for
the force that consumes them, so the quantity here is fixed by its definition. With
A = m^2 - D_eo D_oe (the operator of the CG, conventions of ``oracle.staggered``) and an even-site
field phi, the action is

    S(U) = phi^dagger A(U)^-1 phi.

Moving one link along a traceless Hermitian direction H, U_mu(n) -> exp(i eps H) U_mu(n), changes S
at first order by eps * tr(H G_mu(n)); G_mu(n), a traceless Hermitian 3x3 matrix, is the force.
Differentiating A^-1 and using D_oe = -D_eo^dagger for every gauge field, with x = A^-1 phi (even)
and y = D_oe x (odd):

    dS/deps = 2 Re( x^dagger (dD_eo/deps) y ).

Link U_mu(n) enters D_eo through the forward hop of site n (n even) or the backward hop of site
n + mu (n odd); with c = eta_mu(n) zeta_mu(n) / 2, its hopping coefficient in D,

    n even:  W = c U_mu(n) y(n+mu) x(n)^dagger
    n odd :  W = c y(n) x(n+mu)^dagger U_mu(n)^dagger
    G_mu(n) = i (W - W^dagger)  minus its trace / 3.

Fields are canonical: U complex128[V][4][3][3], x and y complex128[V][3] (only the even half of x
and the odd half of y are read); G is returned as complex128[V][4][3][3].
"""
from __future__ import annotations

import numpy as np

from . import staggered as _st

__all__ = ["fermion_force", "fermion_force_links", "pseudofermion_action_dense", "even_normal_dense"]


def _coeff(dims, mu: int, tbc: float) -> np.ndarray:
    """float64[V]: the hopping coefficient eta_mu(n) zeta_mu(n) / 2 of link U_mu(n) in D."""
    return 0.5 * _st.eta(dims, mu) * _st.zeta(dims, mu, tbc)


def _even_w(c, U, y_fwd, x):
    """W = c U y(n+mu) x(n)^dagger, per site (arrays over sites)."""
    uy = np.einsum("sab,sb->sa", U, y_fwd)
    return c[:, None, None] * np.einsum("sa,sb->sab", uy, np.conj(x))


def _odd_w(c, U, y, x_fwd):
    """W = c y(n) x(n+mu)^dagger U_mu(n)^dagger, per site."""
    yx = np.einsum("sa,sb->sab", y, np.conj(x_fwd))
    return c[:, None, None] * np.einsum("sab,scb->sac", yx, np.conj(U))


def _project(W):
    """i (W - W^dagger) minus its trace / 3 (traceless Hermitian)."""
    G = 1j * (W - np.conj(np.swapaxes(W, -1, -2)))
    tr = np.trace(G, axis1=-2, axis2=-1)
    return G - (tr / 3.0)[..., None, None] * np.eye(3)


def fermion_force(U, x, y, dims, tbc: float = -1.0) -> np.ndarray:
    """G_mu(n) for every link; x even, y odd (the other halves are ignored)."""
    U = np.asarray(U, np.complex128)
    x = np.asarray(x, np.complex128)
    y = np.asarray(y, np.complex128)
    shp = _st._shape4(dims)
    par = _st.parity(dims)
    even = par == 0
    out = np.zeros((U.shape[0], 4, 3, 3), np.complex128)
    for mu in range(4):
        ax = _st._axis(mu)
        c = _coeff(dims, mu, tbc)
        fwd = lambda f: np.roll(f.reshape(shp + f.shape[1:]), -1, axis=ax).reshape(f.shape)  # f(n+mu)
        W_e = _even_w(c, U[:, mu], fwd(y), x)
        W_o = _odd_w(c, U[:, mu], y, fwd(x))
        out[:, mu] = _project(np.where(even[:, None, None], W_e, W_o))
    return out


def fermion_force_links(U, x, y, dims, sites, mus, tbc: float = -1.0) -> np.ndarray:
    """G_mu(n) for listed (site, mu) pairs only (same definition), complex128[len][3][3]."""
    L = [int(d) for d in dims]
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    sites = np.asarray(sites, np.int64)
    mus = np.asarray(mus, np.int64)
    c4 = np.stack([(sites // stride[m]) % L[m] for m in range(4)], axis=1)
    out = np.zeros((len(sites), 3, 3), np.complex128)
    for j, (s, mu) in enumerate(zip(sites, mus)):
        c = c4[j]
        up = s + (((c[mu] + 1) % L[mu]) - c[mu]) * stride[mu]
        eta = -1.0 if c[:mu].sum() % 2 else 1.0
        zeta = tbc if (mu == 3 and c[3] == L[3] - 1) else 1.0
        coef = np.array([0.5 * eta * zeta])
        Uj = np.asarray(U[s, mu])[None]
        if c.sum() % 2 == 0:
            W = _even_w(coef, Uj, np.asarray(y[up])[None], np.asarray(x[s])[None])
        else:
            W = _odd_w(coef, Uj, np.asarray(y[s])[None], np.asarray(x[up])[None])
        out[j] = _project(W)[0]
    return out


def even_normal_dense(U, dims, mass: float, tbc: float = -1.0) -> np.ndarray:
    """The even-site normal operator A = m^2 - D_eo D_oe as a dense matrix on the even sites
    (3 V/2 unknowns; tiny lattices only)."""
    V = _st.volume(dims)
    even = np.nonzero(_st.parity(dims) == 0)[0]
    n = 3 * len(even)
    cols = []
    for j in range(n):
        e = np.zeros((V, 3), np.complex128)
        e[even[j // 3], j % 3] = 1.0
        cols.append(_st.mdagm(U, e, dims, mass, tbc)[even].reshape(-1))
    return np.stack(cols, axis=1)


def pseudofermion_action_dense(U, phi, dims, mass: float, tbc: float = -1.0) -> float:
    """S = phi_e^dagger A^-1 phi_e by a dense LAPACK solve (tiny lattices only)."""
    even = np.nonzero(_st.parity(dims) == 0)[0]
    A = even_normal_dense(U, dims, mass, tbc)
    pe = np.asarray(phi, np.complex128)[even].reshape(-1)
    return float(np.real(np.vdot(pe, np.linalg.solve(A, pe))))
