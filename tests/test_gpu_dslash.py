"""GPU half-lattice operator vs the FP64 oracle, element by element, through the C-ABI."""
import numpy as np
import pytest

from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# several 128-site blocks with a ragged tail, asymmetric extents, the degenerate L = 2 case
SMALL = [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 6, 8), (6, 6, 6, 6), (10, 4, 6, 8), (8, 6, 4, 2)]
ALL_PRECS = ["double", "single18", "single12", "half12", "df64"]


@pytest.fixture(scope="module")
def H():
    from tests import gpu_helpers
    return gpu_helpers


@pytest.mark.parametrize("dims", SMALL)
@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_dslash_all_precisions_match_oracle(H, dims, kind):
    U = I.make_links(dims, kind=kind, seed=1)
    x = I.make_source(dims, seed=3)
    rig = H.Rig(dims, U, precs=ALL_PRECS)
    for par in (0, 1):
        want = S.dslash_parity(U, x, dims, par)
        for name in ALL_PRECS:
            got = rig.dslash(x, par, name)
            assert H.rel(got, want) <= H.TOL[name], (name, par, H.rel(got, want))
            # the other parity's sites of the output are untouched (zero)
            assert np.all(got[S.parity(dims) != par] == 0)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8), (6, 6, 6, 6)])
def test_mdagm_matches_oracle(H, dims):
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=4)
    rig = H.Rig(dims, U, precs=ALL_PRECS)
    for m in (0.5, 0.02):
        want = S.mdagm(U, x, dims, m)
        for name in ALL_PRECS:
            got = rig.mdagm(x, m, name)
            assert H.rel(got, want) <= H.TOL[name], (name, m, H.rel(got, want))


def test_periodic_time_boundary(H):
    dims = (4, 4, 4, 6)
    U = I.make_links(dims, kind="haar", seed=2)
    x = I.make_source(dims, seed=5)
    rig = H.Rig(dims, U, precs=ALL_PRECS, tbc=1)
    for name in ALL_PRECS:
        got = rig.dslash(x, 1, name)
        assert H.rel(got, S.dslash_parity(U, x, dims, 1, tbc=1.0)) <= H.TOL[name]


def test_free_field_closed_form_on_gpu(H):
    """U = 1: (m^2 - D_eo D_oe) on an even plane wave multiplies it by m^2 + sum sin^2 p."""
    dims = (8, 4, 6, 4)
    U = I.make_links(dims, kind="unit")
    rig = H.Rig(dims, U, precs=["double"])
    even = (S.parity(dims) == 0)[:, None]
    k = (1, 1, 2, 3)
    w = np.where(even, I.plane_wave(dims, k, [0.3, 1j, -0.5]), 0.0)
    p = [2 * np.pi * k[mu] / dims[mu] for mu in range(4)]
    p[3] += np.pi / dims[3]
    lam = 0.01 + sum(np.sin(q) ** 2 for q in p)
    assert H.rel(rig.mdagm(w, 0.1), lam * w) <= 1e-13


def test_pack_unpack_round_trip(H):
    import torch
    dims = (6, 4, 2, 4)
    x = I.make_source(dims, seed=8)
    rig = H.Rig(dims, I.make_links(dims, "unit"), precs=["double"])
    xd = H.dev(x)
    for par in (0, 1):
        mask = S.parity(dims) == par
        f = rig.pack(xd, par, 0)
        back = H.host(rig.unpack(f, par, 0))
        assert np.array_equal(back[mask], x[mask])  # bit-exact in FP64
        f = rig.pack(xd, par, 1)
        back = H.host(rig.unpack(f, par, 1))
        assert np.array_equal(back[mask], x[mask].astype(np.complex64).astype(np.complex128))
        f = rig.pack(xd, par, 2)
        back = H.host(rig.unpack(f, par, 2))
        scale = np.max(np.abs(np.stack([x.real, x.imag], -1)), axis=(1, 2))
        err = np.max(np.abs(np.stack([(back - x).real, (back - x).imag], -1)), axis=(1, 2))
        assert np.all(err[mask] <= scale[mask] * 2.0 ** -11 * 1.0001)
        # df64: hi = fl32(v), lo = fl32(v - hi): |error| <= 2^-48 |v| per component
        f = rig.pack(xd, par, 3)
        back = H.host(rig.unpack(f, par, 3))
        assert np.all(np.abs((back - x).real[mask]) <= 2.0 ** -47 * np.abs(x.real[mask]) + 1e-300)
        assert np.all(np.abs((back - x).imag[mask]) <= 2.0 ** -47 * np.abs(x.imag[mask]) + 1e-300)
    del torch


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16])
@pytest.mark.parametrize("name", ["double", "single12", "half12", "df64"])
def test_multi_rhs_matches_oracle(H, nrhs, name):
    dims = (6, 4, 4, 8)
    U = I.make_links(dims, kind="haar", seed=1)
    xs = I.make_sources(dims, nrhs, first_seed=2)
    rig = H.Rig(dims, U, precs=[name])
    got = rig.dslash_mrhs(xs, 1, name)
    for r in range(nrhs):
        assert H.rel(got[r], S.dslash_parity(U, xs[r], dims, 1)) <= H.TOL[name], r


def test_full_size_16_4_double_whole_lattice(H):
    dims = (16, 16, 16, 16)
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "single18", "df64"])
    for par in (0, 1):
        want = S.dslash_parity(U, x, dims, par)
        assert H.rel(rig.dslash(x, par, "double"), want) <= 1e-12
        assert H.rel(rig.dslash(x, par, "single18"), want) <= 1e-5
        assert H.rel(rig.dslash(x, par, "df64"), want) <= 1e-12


def _sample_sites(dims, par, n, seed):
    V = S.volume(dims)
    rng = np.random.default_rng(seed)
    cand = rng.choice(V, size=4 * n, replace=False)
    cand = cand[S.parity_of_sites(dims, cand) == par][:n]
    # always include the lattice corners and the t boundary slices
    edge = np.array([0, V - 1, V // 2, V - V // (dims[3])], np.int64)
    edge = edge[S.parity_of_sites(dims, edge) == par]
    return np.unique(np.concatenate([cand, edge]))


@pytest.mark.parametrize("name", ["double", "single12", "half12", "df64"])
def test_full_size_32_4_sampled_sites(H, name):
    """32^4 (the mixed-precision workload): every output computed, sampled sites checked."""
    dims = (32, 32, 32, 32)
    U = I.make_links(dims, kind="haar", seed=1)
    x = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=[name])
    for par in (0, 1):
        got = rig.dslash(x, par, name)
        sites = _sample_sites(dims, par, 3000, seed=par)
        want = S.dslash_sites(U, x, dims, sites)
        assert H.rel(got[sites], want) <= H.TOL[name], (name, par)
        # properties that hold at any size: other parity untouched, all finite
        assert np.all(got[S.parity_of_sites(dims, np.arange(S.volume(dims))) != par] == 0)
        assert np.all(np.isfinite(got))


def test_full_size_24_4_sixteen_rhs_sampled(H):
    dims = (24, 24, 24, 24)
    U = I.make_links(dims, kind="haar", seed=1)
    xs = I.make_sources(dims, 16, first_seed=2)
    rig = H.Rig(dims, U, precs=["single12"])
    got = rig.dslash_mrhs(xs, 0, "single12")
    sites = _sample_sites(dims, 0, 1000, seed=7)
    for r in range(16):
        assert H.rel(got[r][sites], S.dslash_sites(U, xs[r], dims, sites)) <= 1e-5, r
