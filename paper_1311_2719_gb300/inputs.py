"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only *draws* inputs; it holds none of the Dirac-operator or solver
arithmetic. Every array is produced on the host with NumPy's PCG64 generator so
that both sides of a parity comparison read identical bytes.

Canonical layouts (the public layouts of the C-ABI):
  * site index  i = x0 + L0*(x1 + L1*(x2 + L2*x3)), x3 = t is slowest;
  * links       complex128[V][4][3][3], links[i, mu] = U_mu(n_i) (row-major 3x3);
  * colour field complex128[V][3].

Generators follow the workload recipes of the staggered CG benchmarks:
  * Haar SU(3): complex Gaussian 3x3, QR, the phase of R's diagonal moved into Q
    (so Q is Haar-distributed on U(3)), then Q divided by the principal cube
    root of det Q (det = 1);
  * near-identity SU(3): U = exp(i*eps*H), H = traceless Hermitian part of a
    complex Gaussian matrix, exponentiated through its eigendecomposition;
  * sources: unit-variance complex Gaussian colour vector per site.
"""
from __future__ import annotations

import numpy as np

DIM_NAMES = ("x", "y", "z", "t")


def volume(dims) -> int:
    L0, L1, L2, L3 = (int(d) for d in dims)
    return L0 * L1 * L2 * L3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    g = rng.standard_normal(tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)


def haar_su3(n: int, rng: np.random.Generator) -> np.ndarray:
    """n Haar-random SU(3) matrices, complex128[n][3][3]."""
    z = _complex_gaussian(rng, (n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return np.ascontiguousarray(q)


def near_identity_su3(n: int, rng: np.random.Generator, eps: float) -> np.ndarray:
    """n matrices exp(i*eps*H), H random traceless Hermitian; complex128[n][3][3]."""
    a = _complex_gaussian(rng, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    u = (v * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(v, -1, -2))
    return np.ascontiguousarray(u)


def make_links(dims, kind: str = "haar", seed: int = 1, eps: float = 0.3) -> np.ndarray:
    """Gauge field complex128[V][4][3][3] for the lattice ``dims`` = (L0, L1, L2, L3).

    kind: "haar" (Haar SU(3)), "near_identity" (exp(i eps H)), "unit" (free field).
    """
    V = volume(dims)
    if kind == "unit":
        u = np.zeros((V, 4, 3, 3), np.complex128)
        u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
        return u
    rng = _rng(seed)
    if kind == "haar":
        u = haar_su3(V * 4, rng)
    elif kind == "near_identity":
        u = near_identity_su3(V * 4, rng, eps)
    else:
        raise ValueError(f"unknown link kind {kind!r}")
    return np.ascontiguousarray(u.reshape(V, 4, 3, 3))


def make_source(dims, seed: int = 2) -> np.ndarray:
    """Complex Gaussian colour field complex128[V][3]."""
    return np.ascontiguousarray(_complex_gaussian(_rng(seed), (volume(dims), 3)))


def make_spinor(dims, seed: int = 2) -> np.ndarray:
    """Complex Gaussian Wilson spinor field complex128[V][4][3] (spin, colour)."""
    return np.ascontiguousarray(_complex_gaussian(_rng(seed), (volume(dims), 4, 3)))


def make_sources(dims, nrhs: int, first_seed: int = 2) -> np.ndarray:
    """nrhs sources with seeds first_seed, first_seed+1, ...; complex128[nrhs][V][3]."""
    return np.stack([make_source(dims, first_seed + k) for k in range(nrhs)])


def make_gauge_transform(dims, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per site, complex128[V][3][3]."""
    return haar_su3(volume(dims), _rng(seed))


BATCH_SHAPES = ((4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (8, 8, 8, 16))


def make_lattice_batch(n: int = 64, seed: int = 4, mass_range=(0.02, 0.5)):
    """Uneven batch of independent problems: list of (dims, mass, link_seed, source_seed).

    Shapes are drawn uniformly from {4^4, 6^4, 8^4, 8^3x16}, masses uniformly from
    ``mass_range``; problem j uses link seed 1000+j and source seed 2000+j.
    """
    rng = _rng(seed)
    picks = rng.integers(0, len(BATCH_SHAPES), size=n)
    masses = rng.uniform(mass_range[0], mass_range[1], size=n)
    return [(BATCH_SHAPES[int(p)], float(m), 1000 + j, 2000 + j) for j, (p, m) in enumerate(zip(picks, masses))]


def plane_wave(dims, k, colour, tbc: float = -1.0) -> np.ndarray:
    """exp(i p.n) * colour on every site, p_mu = 2 pi k_mu / L_mu (+ pi/L3 along t when tbc = -1).

    Used only as a test input (a field with a known closed-form image under the free operator).
    """
    L = [int(d) for d in dims]
    x = np.indices((L[3], L[2], L[1], L[0]))  # x[0] = x3, ..., x[3] = x0
    coords = [x[3], x[2], x[1], x[0]]
    phase = np.zeros_like(coords[0], dtype=np.float64)
    for mu in range(4):
        p = 2.0 * np.pi * k[mu] / L[mu]
        if mu == 3 and tbc < 0:
            p += np.pi / L[3]
        phase = phase + p * coords[mu]
    w = np.exp(1j * phase).reshape(-1)
    return np.ascontiguousarray(w[:, None] * np.asarray(colour, np.complex128)[None, :])
