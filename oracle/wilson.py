"""Plain FP64 CPU oracle for the Wilson-fermion operator and its CGNR solve.

TEST INFRASTRUCTURE ONLY: only the test-suite and the benchmark's CPU-baseline leg import it.

The paper's second program (§2: "Wilson fermions with the Wilson gauge action on a single GPU";
§6: its preliminary timings) is only named there. The operator is the standard Wilson hopping
term, written out here by its definition on the full lattice (no even-odd reduction, no spin
projection tricks, dense 4x4 spin matrices):

    D_W psi(n) = sum_mu [ (1 - gamma_mu) zeta_mu(n) U_mu(n) psi(n+mu)
                        + (1 + gamma_mu) zeta_mu(n-mu) U_mu(n-mu)^dagger psi(n-mu) ]
    M = 1 - kappa D_W,     M^dagger = gamma_5 M gamma_5

with zeta = tbc (-1, antiperiodic) on the t-links of the last time slice, and the gamma matrices
of the DeGrand-Rossi basis (index order mu = x, y, z, t). Fields are complex128[V][4][3]
(spin, colour), links complex128[V][4][3][3], site order as in the staggered oracle.
"""
from __future__ import annotations

import numpy as np

from . import staggered as _st

# DeGrand-Rossi gamma matrices, mu = 0..3 = x, y, z, t (Hermitian, {g_mu, g_nu} = 2 delta)
GAMMA = np.array([
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
EYE4 = np.eye(4, dtype=np.complex128)


def dslash_w(U, psi, dims, tbc: float = -1.0) -> np.ndarray:
    """Full-lattice Wilson hopping term D_W psi (complex128[V][4][3])."""
    shp = _st._shape4(dims)
    U4 = np.asarray(U, np.complex128).reshape(shp + (4, 3, 3))
    p4 = np.asarray(psi, np.complex128).reshape(shp + (4, 3))
    out = np.zeros_like(p4)
    for mu in range(4):
        ax = _st._axis(mu)
        z = _st.zeta(dims, mu, tbc).reshape(shp)
        link = U4[..., mu, :, :] * z[..., None, None]
        fwd = np.einsum("...ab,...sb->...sa", link, np.roll(p4, -1, axis=ax))          # U psi(n+mu)
        fwd = np.einsum("st,...ta->...sa", EYE4 - GAMMA[mu], fwd)                       # (1 - g_mu)
        link_b = np.roll(link, 1, axis=ax)                                             # U(n-mu)
        bwd = np.einsum("...ba,...sb->...sa", np.conj(link_b), np.roll(p4, 1, axis=ax))  # U^dagger psi(n-mu)
        bwd = np.einsum("st,...ta->...sa", EYE4 + GAMMA[mu], bwd)                       # (1 + g_mu)
        out += fwd + bwd
    return out.reshape(-1, 4, 3)


def gamma5(psi) -> np.ndarray:
    return np.einsum("st,...ta->...sa", GAMMA5, np.asarray(psi, np.complex128))


def apply_m(U, psi, dims, kappa: float, tbc: float = -1.0) -> np.ndarray:
    """M psi = psi - kappa D_W psi."""
    return np.asarray(psi, np.complex128) - kappa * dslash_w(U, psi, dims, tbc)


def apply_mdag(U, psi, dims, kappa: float, tbc: float = -1.0) -> np.ndarray:
    """M^dagger psi = gamma5 M gamma5 psi."""
    return gamma5(apply_m(U, gamma5(psi), dims, kappa, tbc))


def _n2(a) -> float:
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def cgnr(U, b, dims, kappa: float, tol: float, max_iter: int, tbc: float = -1.0):
    """CG on the normal equations M^dagger M x = M^dagger b (textbook order: x = 0, r = p = M^dagger b,
    alpha = |r|^2 / |M p|^2, x += alpha p, r -= alpha M^dagger M p, beta = |r_new|^2 / |r|^2).

    Stops when |r|^2 < tol^2 |M^dagger b|^2. Returns dict(x, iterations, converged,
    normal_rel_residual = |M^dagger b - M^dagger M x| / |M^dagger b|, rel_residual = |b - M x| / |b|).
    """
    b = np.asarray(b, np.complex128)
    rhs = apply_mdag(U, b, dims, kappa, tbc)
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = _n2(r)
    stop = tol * tol * _n2(rhs)
    it = 0
    while rr >= stop and it < max_iter:
        t = apply_m(U, p, dims, kappa, tbc)
        alpha = rr / _n2(t)
        x = x + alpha * p
        r = r - alpha * apply_mdag(U, t, dims, kappa, tbc)
        rr_new = _n2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    out = {"x": x, "iterations": it, "converged": rr < stop}
    out.update(residuals(U, x, b, dims, kappa, tbc))
    return out


def residuals(U, x, b, dims, kappa: float, tbc: float = -1.0) -> dict:
    """The two FP64 residuals of a solution x of M x = b: rel_residual = |b - M x| / |b| and
    normal_rel_residual = |M^dagger b - M^dagger M x| / |M^dagger b| (the CGNR's own system)."""
    b = np.asarray(b, np.complex128)
    rhs = apply_mdag(U, b, dims, kappa, tbc)
    nres = rhs - apply_mdag(U, apply_m(U, x, dims, kappa, tbc), dims, kappa, tbc)
    res = b - apply_m(U, x, dims, kappa, tbc)
    return {"normal_rel_residual": float(np.sqrt(_n2(nres) / _n2(rhs))),
            "rel_residual": float(np.sqrt(_n2(res) / _n2(b)))}


def dslash_w_sites(U, psi, dims, sites, tbc: float = -1.0) -> np.ndarray:
    """D_W psi at the listed canonical sites only (same definition), complex128[len(sites)][4][3]."""
    L = [int(d) for d in dims]
    stride = [1, L[0], L[0] * L[1], L[0] * L[1] * L[2]]
    sites = np.asarray(sites, np.int64)
    c = np.stack([(sites // stride[mu]) % L[mu] for mu in range(4)], axis=1)
    U = np.asarray(U)
    psi = np.asarray(psi)
    out = np.zeros((len(sites), 4, 3), np.complex128)
    for mu in range(4):
        up = sites + (((c[:, mu] + 1) % L[mu]) - c[:, mu]) * stride[mu]
        dn = sites + (((c[:, mu] - 1) % L[mu]) - c[:, mu]) * stride[mu]
        z_f = np.where((mu == 3) & (c[:, 3] == L[3] - 1), tbc, 1.0)
        z_b = np.where((mu == 3) & (c[:, 3] == 0), tbc, 1.0)
        f = np.einsum("sab,stb->sta", U[sites, mu], psi[up]) * z_f[:, None, None]
        bk = np.einsum("sba,stb->sta", np.conj(U[dn, mu]), psi[dn]) * z_b[:, None, None]
        out += np.einsum("uv,svb->sub", EYE4 - GAMMA[mu], f) + np.einsum("uv,svb->sub", EYE4 + GAMMA[mu], bk)
    return out
