"""Plain FP64 CPU oracle for the staggered Dirac operator and its even-odd CG solve.

TEST INFRASTRUCTURE ONLY. This module is the correctness reference for the CUDA
path: only the test-suite, the smoke check and the benchmark's CPU-baseline leg
may import it. The library never calls it and never falls back to it.

It is deliberately slow and literal: every function works on full-lattice
canonical arrays (site index i = x0 + L0*(x1 + L1*(x2 + L2*x3)), links
complex128[V][4][3][3], colour fields complex128[V][3]), computes neighbours by
rolling the 4-D array, and applies the staggered phases from the coordinates.
No even-odd packing, no folded phases, no neighbour tables, no fusion.

Conventions (the paper leaves them unstated; these are the readings adopted):
  * eta_mu(n)  = (-1)^(x0 + ... + x_{mu-1})            (eta_0 = 1)
  * zeta_mu(n) = tbc (= -1, antiperiodic) on the t-links U_3(n) with x3 = L3-1, else +1
  * D x(n) = 1/2 sum_mu [ eta_mu(n) zeta_mu(n) U_mu(n) x(n+mu)
                          - eta_mu(n-mu) zeta_mu(n-mu) U_mu(n-mu)^dagger x(n-mu) ]
    so D is anti-Hermitian and M = m + D has M^dagger M = m^2 - D^2;
  * even-odd: parity(n) = (x0+x1+x2+x3) mod 2; D maps each parity onto the other,
    D_eo: odd -> even, D_oe: even -> odd, and the even-site normal operator is
    A = m^2 - D_eo D_oe = m^2 + D_oe^dagger D_oe.

Paper passages followed: §3 (the matrix-vector routine: a site loop that gathers
the forward and backward neighbours through iup/idn and multiplies by the links
u and their conjugates ud) and §4 (the single-GPU congrad listing: CG on the
even-parity normal equations with x = 0, p = r = b, alpha's denominator
<Kp,Kp> + <p,p>, the fermion-matrix-transpose step, the betan < delit exit test
and the final opposite-parity image y = K x).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume", "coords", "parity", "eta", "zeta", "dslash", "dslash_parity",
    "mdagm", "cg_solve", "true_residual", "neighbour_tables", "dense_operator",
    "reconstruct_third_row",
]


def volume(dims) -> int:
    L0, L1, L2, L3 = (int(d) for d in dims)
    return L0 * L1 * L2 * L3


def _shape4(dims):
    """numpy shape of a lattice array: (L3, L2, L1, L0) so that x0 is fastest."""
    L0, L1, L2, L3 = (int(d) for d in dims)
    return (L3, L2, L1, L0)


def _axis(mu: int) -> int:
    """numpy axis of lattice direction mu in the (L3, L2, L1, L0) view."""
    return 3 - mu


def coords(dims) -> np.ndarray:
    """int64[V][4]: (x0, x1, x2, x3) of every site in canonical order."""
    g = np.indices(_shape4(dims)).reshape(4, -1)  # g[0] = x3, ..., g[3] = x0
    return np.stack([g[3], g[2], g[1], g[0]], axis=1)


def parity(dims) -> np.ndarray:
    """int64[V]: (x0+x1+x2+x3) mod 2."""
    return coords(dims).sum(axis=1) % 2


def eta(dims, mu: int) -> np.ndarray:
    """float64[V]: staggered phase eta_mu(n) = (-1)^(x0+...+x_{mu-1})."""
    c = coords(dims)
    return np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0)


def zeta(dims, mu: int, tbc: float = -1.0) -> np.ndarray:
    """float64[V]: boundary sign carried by the link U_mu(n): tbc on the last t-slice for mu = 3."""
    z = np.ones(volume(dims))
    if mu == 3:
        z[coords(dims)[:, 3] == int(dims[3]) - 1] = tbc
    return z


def dslash(U: np.ndarray, x: np.ndarray, dims, tbc: float = -1.0) -> np.ndarray:
    """Full-lattice staggered hopping term D x (paper §3, the matrix-vector routine).

    U: complex128[V][4][3][3], x: complex128[V][3]; returns complex128[V][3].
    Forward hop: eta*zeta*U_mu(n) x(n+mu). Backward hop: the same phased link taken
    at n-mu, daggered, times x(n-mu), with a minus sign. Overall factor 1/2.
    """
    shp = _shape4(dims)
    U4 = np.asarray(U, np.complex128).reshape(shp + (4, 3, 3))
    x4 = np.asarray(x, np.complex128).reshape(shp + (3,))
    out = np.zeros_like(x4)
    for mu in range(4):
        ax = _axis(mu)
        s = (eta(dims, mu) * zeta(dims, mu, tbc)).reshape(shp)
        link = U4[..., mu, :, :] * s[..., None, None]          # phased U_mu(n)
        x_fwd = np.roll(x4, -1, axis=ax)                       # x(n+mu)
        fwd = np.einsum("...ab,...b->...a", link, x_fwd)
        link_bwd = np.roll(link, 1, axis=ax)                   # phased U_mu(n-mu)
        x_bwd = np.roll(x4, 1, axis=ax)                        # x(n-mu)
        bwd = np.einsum("...ba,...b->...a", np.conj(link_bwd), x_bwd)  # U^dagger x
        out += 0.5 * (fwd - bwd)
    return out.reshape(-1, 3)


def dslash_parity(U, x, dims, out_parity: int, tbc: float = -1.0) -> np.ndarray:
    """D restricted to one output parity: out = D x on sites of ``out_parity``, 0 elsewhere.

    Only the opposite-parity half of ``x`` contributes (D connects the two parities);
    this is the half-lattice form the paper's fmv / fmtv calls apply (paper §4).
    """
    par = parity(dims)
    xin = np.where((par != out_parity)[:, None], x, 0.0)
    out = dslash(U, xin, dims, tbc)
    return np.where((par == out_parity)[:, None], out, 0.0)


def mdagm(U, x, dims, mass: float, tbc: float = -1.0) -> np.ndarray:
    """Even-site normal operator A x_e = m^2 x_e - D_eo D_oe x_e; the odd half of the result is 0.

    Built by running the full operator twice on the even-supported vector, as the
    definition M^dagger M = m^2 - D^2 restricted to even sites states.
    """
    par = parity(dims)
    xe = np.where((par == 0)[:, None], x, 0.0)
    d2 = dslash(U, dslash(U, xe, dims, tbc), dims, tbc)
    out = mass * mass * xe - d2
    return np.where((par == 0)[:, None], out, 0.0)


def _dot(a, b) -> complex:
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def _norm2(a) -> float:
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def cg_solve(U, b, dims, mass: float, tol: float, max_iter: int, tbc: float = -1.0):
    """Conjugate gradient on the even-site normal equations, in the order of the paper's congrad (§4).

    b: complex128[V][3] (only its even half is used). Stops when <r,r> < delit with
    delit = tol^2 <b_e,b_e> (a relative residual tol), or after max_iter iterations.
    Returns dict(x=even solution (odd half 0), y = D_oe x on odd sites, iterations,
    converged, true_rel_residual = |b_e - A x| / |b_e| recomputed after the loop).
    """
    par = parity(dims)
    even = (par == 0)[:, None]
    odd = (par == 1)[:, None]
    m2 = mass * mass
    be = np.where(even, np.asarray(b, np.complex128), 0.0)
    x = np.zeros_like(be)
    r = be.copy()
    p = be.copy()
    betan = _norm2(r)
    delit = tol * tol * _norm2(be)
    iters = 0
    converged = betan < delit
    alphan = betan
    while not converged and iters < max_iter:
        iters += 1
        ap = np.where(odd, dslash(U, p, dims, tbc), 0.0)           # ap = K p   (K = D_oe)
        alphad = _norm2(ap) + m2 * _norm2(p)                        # <Kp,Kp> + m^2 <p,p>
        alpha = alphan / alphad
        x = x + alpha * p
        atap = m2 * p - np.where(even, dslash(U, ap, dims, tbc), 0.0)  # m^2 p + K^dagger K p
        r = r - alpha * atap
        betan_new = _norm2(r)
        if betan_new < delit:
            converged = True
            break
        beta = betan_new / alphan
        alphan = betan_new
        p = r + beta * p
    y = np.where(odd, dslash(U, x, dims, tbc), 0.0)                 # y = K x on the odd sites
    return {
        "x": x,
        "y": y,
        "iterations": iters,
        "converged": bool(converged),
        "true_rel_residual": true_residual(U, x, be, dims, mass, tbc),
    }


def true_residual(U, x, b, dims, mass: float, tbc: float = -1.0) -> float:
    """|b_e - A x_e| / |b_e| in FP64."""
    par = parity(dims)
    be = np.where((par == 0)[:, None], b, 0.0)
    res = be - mdagm(U, x, dims, mass, tbc)
    return float(np.sqrt(_norm2(res) / _norm2(be)))


def neighbour_tables(dims):
    """Canonical neighbour tables, int64[V][4]: iup[i, mu] = index of n+mu, idn[i, mu] = index of n-mu.

    These are the paper's iup/idn arrays (§3), written out from the coordinates.
    """
    L = [int(d) for d in dims]
    c = coords(dims)
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    V = volume(dims)
    iup = np.zeros((V, 4), np.int64)
    idn = np.zeros((V, 4), np.int64)
    base = np.arange(V)
    for mu in range(4):
        up = (c[:, mu] + 1) % L[mu]
        dn = (c[:, mu] - 1) % L[mu]
        iup[:, mu] = base + (up - c[:, mu]) * stride[mu]
        idn[:, mu] = base + (dn - c[:, mu]) * stride[mu]
    return iup, idn


def dense_operator(apply, n_sites: int) -> np.ndarray:
    """Brute-force matrix of a linear map on colour fields: column j = apply(e_j). For tiny lattices."""
    n = 3 * n_sites
    cols = []
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        cols.append(np.asarray(apply(e.reshape(n_sites, 3))).reshape(-1))
    return np.stack(cols, axis=1)


def reconstruct_third_row(a, b) -> np.ndarray:
    """Third row of an SU(3) matrix from its first two rows: c = conj(a x b) (unitarity + det = 1).

    This is the identity behind storing two rows of each link (the paper's remark in §6 on keeping
    only part of the gauge field).
    """
    a = np.asarray(a)
    b = np.asarray(b)
    return np.conj(np.cross(a, b))


def dslash_sites(U, x, dims, sites, tbc: float = -1.0) -> np.ndarray:
    """D x evaluated at the listed canonical sites only (same definition as ``dslash``).

    For checks on lattices too large for the full-lattice oracle: each site's value is
    computed from its own coordinates, its 8 neighbours and the 8 links that touch it.
    Returns complex128[len(sites)][3].
    """
    L = [int(d) for d in dims]
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    sites = np.asarray(sites, np.int64)
    c = np.stack([(sites // stride[mu]) % L[mu] for mu in range(4)], axis=1)
    U = np.asarray(U)
    x = np.asarray(x)
    out = np.zeros((len(sites), 3), np.complex128)
    for mu in range(4):
        eta_n = np.where(c[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0)
        up = sites + (((c[:, mu] + 1) % L[mu]) - c[:, mu]) * stride[mu]
        dn = sites + (((c[:, mu] - 1) % L[mu]) - c[:, mu]) * stride[mu]
        z_fwd = np.where((mu == 3) & (c[:, 3] == L[3] - 1), tbc, 1.0)
        z_bwd = np.where((mu == 3) & (c[:, 3] == 0), tbc, 1.0)   # the link U_3(n-3) sits on x3 = L3-1
        fwd = np.einsum("sab,sb->sa", U[sites, mu], x[up])
        bwd = np.einsum("sba,sb->sa", np.conj(U[dn, mu]), x[dn])
        out += 0.5 * eta_n[:, None] * (z_fwd[:, None] * fwd - z_bwd[:, None] * bwd)
    return out


def mdagm_sites(U, x, dims, mass: float, sites, tbc: float = -1.0) -> np.ndarray:
    """(A x)(n) = m^2 x(n) - (D D x_e)(n) at the listed even sites; x is a full canonical field.

    Only the even half of x is used. Builds D x_e at the neighbours of the sites, then D of that.
    """
    dims = tuple(int(d) for d in dims)
    sites = np.asarray(sites, np.int64)
    par = parity_of_sites(dims, sites)
    if np.any(par != 0):
        raise ValueError("mdagm_sites takes even sites")
    xe = np.array(x, np.complex128, copy=True)
    xe[parity_of_sites(dims, np.arange(volume(dims))) == 1] = 0.0
    iup, idn = neighbour_tables_of_sites(dims, sites)
    nb = np.unique(np.concatenate([iup.reshape(-1), idn.reshape(-1)]))
    y = np.zeros_like(xe)
    y[nb] = dslash_sites(U, xe, dims, nb, tbc)
    return mass * mass * xe[sites] - dslash_sites(U, y, dims, sites, tbc)


def parity_of_sites(dims, sites) -> np.ndarray:
    L = [int(d) for d in dims]
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    sites = np.asarray(sites, np.int64)
    return sum((sites // stride[mu]) % L[mu] for mu in range(4)) % 2


def neighbour_tables_of_sites(dims, sites):
    """iup/idn rows (int64[len(sites)][4]) for the listed canonical sites."""
    L = [int(d) for d in dims]
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    sites = np.asarray(sites, np.int64)
    iup = np.zeros((len(sites), 4), np.int64)
    idn = np.zeros((len(sites), 4), np.int64)
    for mu in range(4):
        c = (sites // stride[mu]) % L[mu]
        iup[:, mu] = sites + (((c + 1) % L[mu]) - c) * stride[mu]
        idn[:, mu] = sites + (((c - 1) % L[mu]) - c) * stride[mu]
    return iup, idn


def apply_m(U, x, dims, mass: float, tbc: float = -1.0) -> np.ndarray:
    """The full staggered operator M x = m x + D x on both parities."""
    return mass * np.asarray(x, np.complex128) + dslash(U, x, dims, tbc)


def solve_full(U, b, dims, mass: float, tol: float, max_iter: int, tbc: float = -1.0):
    """x = M^-1 b on the full lattice, M = m + D.

    Textbook CG on the normal equations M^dagger M x = M^dagger b, with M^dagger = m - D (D is
    anti-Hermitian) and M^dagger M = m^2 - D^2, over both parities at once; no even-odd
    reduction. Stops when |M^dagger b - M^dagger M x| <= tol |M^dagger b|.
    Returns dict(x, iterations, rel_residual = |b - M x| / |b|).
    """
    b = np.asarray(b, np.complex128)
    rhs = mass * b - dslash(U, b, dims, tbc)

    def normal(v):
        return mass * mass * v - dslash(U, dslash(U, v, dims, tbc), dims, tbc)

    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = _norm2(r)
    stop = tol * tol * _norm2(rhs)
    it = 0
    while rr > stop and it < max_iter:
        ap = normal(p)
        alpha = rr / float(np.vdot(p.reshape(-1), ap.reshape(-1)).real)
        x = x + alpha * p
        r = r - alpha * ap
        rr_new = _norm2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return {"x": x, "iterations": it, "rel_residual": full_residual(U, x, b, dims, mass, tbc)}


def full_residual(U, x, b, dims, mass: float, tbc: float = -1.0) -> float:
    """|b - M x| / |b| in FP64 over both parities, M = m + D."""
    b = np.asarray(b, np.complex128)
    res = b - apply_m(U, x, dims, mass, tbc)
    return float(np.sqrt(_norm2(res) / _norm2(b)))
