"""GPU half-lattice operator vs the FP64 oracle, element by element, through the C-ABI."""
import numpy as np
import pytest

from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I
from paper_1311_2719_gb300 import qcd as Q

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


# ---- the 16-bit formats, written out from their definitions (test-side; the oracle is FP64)
def _fx16(v):
    """16-bit fixed-point code of reals |v| <= 1: round(fl32(v) * 2^15) + 2^15, saturated to 16 bits."""
    t = np.rint(np.asarray(v).astype(np.float32) * np.float32(32768.0))
    return (np.clip(t, -32768.0, 32767.0).astype(np.int64) + 32768).astype(np.uint32)


def _eo_lex(dims, par):
    """Canonical index of even-odd site k (k = 0 .. V/2-1) of parity `par`: the canonical pair
    (2k, 2k+1) shares x1..x3 and holds one site of each parity."""
    L0, L1, L2, _ = dims
    j = 2 * np.arange(int(np.prod(dims)) // 2)
    x0e, t = j % L0, j // L0
    x1, t1 = t % L1, t // L1
    x2, x3 = t1 % L2, t1 // L2
    return j + ((x1 + x2 + x3 + par) & 1)


def _half_field(x):
    """A canonical field quantised as the 16-bit vector format stores it: per site m = max |re|, |im|
    over the colours (FP32), each component fl16(fl32(v) * fl32(1 / m)), read back as that times m."""
    re, im = x.real.astype(np.float32), x.imag.astype(np.float32)
    m = np.maximum(np.abs(re).max(axis=1), np.abs(im).max(axis=1))
    inv = np.where(m > 0, np.float32(1.0) / np.where(m > 0, m, np.float32(1.0)), np.float32(0.0)).astype(np.float32)
    qr = (re * inv[:, None]).astype(np.float16).astype(np.float64)
    qi = (im * inv[:, None]).astype(np.float16).astype(np.float64)
    return (qr + 1j * qi) * m.astype(np.float64)[:, None], m.astype(np.float64)


def test_fixed_point_links_are_bit_exact(H):
    """QCD_PREC_HALF recon-12 links are integer data: each 32-bit word is the (re, im) pair of one
    element of rows 0 and 1 in 16-bit fixed point, laid out [parity][mu][site] as four words
    (elements 00 01 02 10) and then, after all of them, two words (11 12)."""
    dims = (4, 6, 2, 8)
    U = I.make_links(dims, kind="haar", seed=3)
    U[5, 2] = np.eye(3)    # elements 1 and 0: the saturated code and the bias
    U[7, 1] = -np.eye(3)   # -1: the lowest code
    rig = H.Rig(dims, U, precs=[])
    words = H.host(rig.lat.load_links(rig.U_dev, Q.QCD_PREC_HALF, 12)).view(np.uint32)
    Vh = U.shape[0] // 2
    assert words.size == 8 * Vh * 6
    A = words[: 8 * Vh * 4].reshape(2, 4, Vh, 4)
    B = words[8 * Vh * 4:].reshape(2, 4, Vh, 2)
    for par in (0, 1):
        E = U[_eo_lex(dims, par)][:, :, :2, :].reshape(Vh, 4, 6)
        W = (_fx16(E.real) | (_fx16(E.imag) << np.uint32(16))).transpose(1, 0, 2)
        assert np.array_equal(A[par], W[..., :4]) and np.array_equal(B[par], W[..., 4:]), par


@pytest.mark.parametrize("dims,out_par", [((4, 6, 2, 8), 1), ((6, 4, 4, 4), 0)])
def test_16bit_operator_matches_oracle_on_its_quantised_inputs(H, dims, out_par):
    """The 16-bit operator, fed links and a vector that are exact in its formats, differs from the
    FP64 oracle on the same quantised inputs by FP32 arithmetic and the output's FP16 rounding only:
    per site at most 2^-11 of the site's largest component (half an FP16 step is 2^-12)."""
    U = I.make_links(dims, kind="haar", seed=5)
    x = I.make_source(dims, seed=6)
    Uq = U.copy()
    rows = _fx16(np.stack([U[:, :, :2, :].real, U[:, :, :2, :].imag], -1)).astype(np.float64)
    deq = (rows - 32768.0) / 32768.0
    Uq[:, :, :2, :] = deq[..., 0] + 1j * deq[..., 1]
    a, b = Uq[:, :, 0, :], Uq[:, :, 1, :]
    Uq[:, :, 2, :] = np.conj(np.cross(a, b))  # the third row as every recon-12 kernel rebuilds it
    rig = H.Rig(dims, U, precs=["half12"])
    xin = np.where((S.parity(dims) != out_par)[:, None], _half_field(x)[0], 0.0)
    want = S.dslash_parity(Uq, xin, dims, out_par)
    got = rig.dslash(xin, out_par, "half12")
    sites = S.parity(dims) == out_par
    m = np.max(np.abs(np.stack([want.real, want.imag], -1)), axis=(1, 2))
    err = np.max(np.abs(np.stack([(got - want).real, (got - want).imag], -1)), axis=(1, 2))
    assert np.all(err[sites] <= 2.0 ** -11 * m[sites]), float(np.max(err[sites] / m[sites]))
    assert np.all(got[~sites] == 0)
