"""GPU Wilson operator and CGNR vs the FP64 Wilson oracle, through the C-ABI."""
import numpy as np
import pytest

from oracle import staggered as S
from oracle import wilson as W
from paper_1311_2719_gb300 import inputs as I
from paper_1311_2719_gb300 import qcd as Q

pytestmark = pytest.mark.gpu

TOL = {Q.QCD_PREC_DOUBLE: 1e-12, Q.QCD_PREC_SINGLE: 1e-5}


@pytest.fixture(scope="module")
def H():
    from tests import gpu_helpers
    return gpu_helpers


class WRig:
    def __init__(self, H, dims, U, precs=(Q.QCD_PREC_DOUBLE, Q.QCD_PREC_SINGLE)):
        import torch
        self.torch, self.H = torch, H
        self.dims = dims
        self.lat = Q.Lattice(dims)
        self.h = self.lat.handle
        self.V = self.lat.V
        self.Ud = H.dev(U)
        self.links = {}
        for p in precs:
            buf = self.lat.empty_bytes(Q.qcd_wilson_links_bytes(self.h, p))
            Q.qcd_wilson_load_links(self.h, self.Ud, buf, p)
            self.links[p] = buf

    def field(self, prec):
        return self.lat.empty_bytes(Q.qcd_wilson_field_bytes(self.h, prec))

    def op(self, psi, kappa, op, prec):
        fin, fout = self.field(prec), self.field(prec)
        Q.qcd_wilson_pack_field(self.h, fin, self.H.dev(psi), prec)
        Q.qcd_wilson_op(self.h, fout, fin, kappa, op, prec)
        out = self.torch.zeros((self.V, 4, 3), dtype=self.torch.complex128, device="cuda")
        Q.qcd_wilson_unpack_field(self.h, out, fout, prec)
        return self.H.host(out)

    def cgnr(self, b, kappa, tol=1e-10, prec=Q.QCD_PREC_DOUBLE, max_iter=10000):
        opts = Q.qcd_solver_opts_default()
        opts.prec_inner = prec
        ws = self.lat.empty_bytes(Q.qcd_wilson_workspace_bytes(self.h, opts))
        bd = self.H.dev(b)
        x = self.torch.zeros_like(bd)
        s = self.torch.cuda.Stream()
        s.wait_stream(self.torch.cuda.current_stream())
        rc, info = Q.qcd_wilson_cgnr(self.h, x, bd, kappa, tol, max_iter, opts, ws, stream=s)
        s.synchronize()
        return rc, info, self.H.host(x)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 6, 8), (6, 4, 2, 4), (4, 6, 4, 10)])
def test_wilson_operators_match_oracle(H, dims):
    U = I.make_links(dims, kind="haar", seed=1)
    psi = I.make_spinor(dims, seed=3)
    rig = WRig(H, dims, U)
    kappa = 0.125
    want = {Q.QCD_WILSON_DSLASH: W.dslash_w(U, psi, dims), Q.QCD_WILSON_M: W.apply_m(U, psi, dims, kappa),
            Q.QCD_WILSON_MDAG: W.apply_mdag(U, psi, dims, kappa)}
    for prec in (Q.QCD_PREC_DOUBLE, Q.QCD_PREC_SINGLE):
        for op, w in want.items():
            got = rig.op(psi, kappa, op, prec)
            assert H.rel(got, w) <= TOL[prec], (prec, op, H.rel(got, w))


def test_wilson_free_field_closed_form_on_gpu(H):
    dims = (4, 6, 4, 8)
    U = I.make_links(dims, kind="unit")
    rig = WRig(H, dims, U, precs=(Q.QCD_PREC_DOUBLE,))
    kappa = 0.11
    k = (1, 2, 3, 5)
    psi0 = np.arange(12).reshape(4, 3) * (0.3 + 0.1j) + 1.0
    phase = I.plane_wave(dims, k, [1.0, 0, 0])[:, 0]
    psi = phase[:, None, None] * psi0[None]
    p = [2 * np.pi * k[mu] / dims[mu] for mu in range(4)]
    p[3] += np.pi / dims[3]
    Mp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(W.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    want = phase[:, None, None] * (Mp @ psi0)[None]
    assert H.rel(rig.op(psi, kappa, Q.QCD_WILSON_M, Q.QCD_PREC_DOUBLE), want) <= 1e-13


def test_wilson_pack_round_trip(H):
    import torch
    dims = (4, 2, 6, 2)
    psi = I.make_spinor(dims, seed=8)
    rig = WRig(H, dims, I.make_links(dims, "unit"), precs=(Q.QCD_PREC_DOUBLE,))
    for prec in (Q.QCD_PREC_DOUBLE, Q.QCD_PREC_SINGLE):
        f = rig.field(prec)
        Q.qcd_wilson_pack_field(rig.h, f, H.dev(psi), prec)
        back = torch.zeros((rig.V, 4, 3), dtype=torch.complex128, device="cuda")
        Q.qcd_wilson_unpack_field(rig.h, back, f, prec)
        want = psi if prec == Q.QCD_PREC_DOUBLE else psi.astype(np.complex64).astype(np.complex128)
        assert np.array_equal(H.host(back), want)


@pytest.mark.parametrize("prec", [Q.QCD_PREC_DOUBLE, Q.QCD_PREC_SINGLE])
@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.125), ((2, 4, 6, 8), 0.14), ((6, 6, 4, 4), 0.1)])
def test_wilson_cgnr_matches_oracle(H, prec, dims, kappa):
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_spinor(dims, seed=2)
    rig = WRig(H, dims, U)
    rc, info, x = rig.cgnr(b, kappa, 1e-10, prec)
    assert rc == Q.QCD_OK, info
    assert info["true_rel_residual"] <= 1e-10
    rhs = W.apply_mdag(U, b, dims, kappa)
    nres = rhs - W.apply_mdag(U, W.apply_m(U, x, dims, kappa), dims, kappa)
    assert np.linalg.norm(nres) / np.linalg.norm(rhs) <= 1.01e-10
    ref = W.cgnr(U, b, dims, kappa, tol=1e-12, max_iter=10000)
    assert H.rel(x, ref["x"]) <= 1e-7
    if prec == Q.QCD_PREC_SINGLE:
        assert info["reliable_updates"] >= 1


def test_wilson_status_codes(H):
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="haar", seed=1)
    rig = WRig(H, dims, U)
    b = I.make_spinor(dims, seed=2)
    rc, info, _ = rig.cgnr(b, 0.125, max_iter=3)
    assert rc == Q.QCD_ERR_NOT_CONVERGED and info["iterations"] == 3
    bn = b.copy()
    bn[7, 1, 2] = np.nan
    rc, info, _ = rig.cgnr(bn, 0.125)
    assert rc == Q.QCD_ERR_BREAKDOWN
    rc, info, x = rig.cgnr(np.zeros_like(b), 0.125)
    assert rc == Q.QCD_OK and not np.any(x)


def test_wilson_full_size_32c64(H):
    """32^3 x 64, kappa = 0.125, Haar links: sampled-site operator parity and a mixed CGNR to 1e-10."""
    dims = (32, 32, 32, 64)
    kappa = 0.125
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_spinor(dims, seed=2)
    rig = WRig(H, dims, U)
    V = S.volume(dims)
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([rng.choice(V, 1500, replace=False), [0, V - 1, V // 2]]))
    for prec in (Q.QCD_PREC_DOUBLE, Q.QCD_PREC_SINGLE):
        got = rig.op(b, kappa, Q.QCD_WILSON_DSLASH, prec)
        assert H.rel(got[sites], W.dslash_w_sites(U, b, dims, sites)) <= TOL[prec]
    rc, info, x = rig.cgnr(b, kappa, 1e-10, Q.QCD_PREC_SINGLE)
    assert rc == Q.QCD_OK and info["true_rel_residual"] <= 1e-10
