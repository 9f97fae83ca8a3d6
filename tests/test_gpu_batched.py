"""Batched solves on the GPU: multi-RHS CG on one lattice and the persistent multi-lattice CG,
checked against the FP64 oracle, against the single-RHS solver, and for their status codes."""
import os
import tempfile

import numpy as np
import pytest

from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I
from paper_1311_2719_gb300 import qcd as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from tests import gpu_helpers
    return gpu_helpers


def _kappa(m):
    return (m * m + 16.0) / (m * m)


def _mrhs(H, rig, bs, mass, inner="double", rb=0, tol=1e-10, max_iter=20000, want_y=True):
    import torch
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = H.PRECS[inner]
    opts.rhs_block = rb
    n = len(bs)
    ws = rig.lat.workspace(opts, n)
    bd = H.dev(np.stack(bs))
    x = torch.zeros_like(bd)
    y = torch.zeros_like(bd) if want_y else None
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rc, infos = Q.qcd_cg_solve_mrhs(rig.h, n, x, bd, mass, tol, max_iter, opts, ws, y, stream=s)
    s.synchronize()
    return rc, infos, H.host(x), (H.host(y) if want_y else None)


@pytest.mark.parametrize("inner", ["double", "single12", "half12", "df64"])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_mrhs_cg_matches_oracle(H, inner, nrhs):
    dims, m = (6, 4, 4, 8), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    bs = list(I.make_sources(dims, nrhs, first_seed=2))
    rig = H.Rig(dims, U, precs=sorted({"double", inner}))
    rc, infos, x, y = _mrhs(H, rig, bs, m, inner)
    assert rc == Q.QCD_OK, infos
    for r in range(nrhs):
        assert infos[r]["converged"] and infos[r]["true_rel_residual"] <= 1e-10
        assert S.true_residual(U, x[r], bs[r], dims, m) <= 1.01e-10
        ref = S.cg_solve(U, bs[r], dims, m, tol=1e-12, max_iter=5000)
        assert H.rel(x[r], ref["x"]) <= _kappa(m) * 1e-10
        assert H.rel(y[r], S.dslash_parity(U, x[r], dims, 1)) <= 1e-12


@pytest.mark.parametrize("inner", ["double", "single12", "half12", "df64"])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 4, 8), 3), ((10, 4, 6, 8), 9), ((8, 8, 8, 8), 16)])
def test_mrhs_shared_link_kernel_matches_oracle(H, inner, dims, nrhs):
    """The shared-link multi-RHS operator (rhs_block = -1): tiles of 32 sites with a ragged last
    tile (10x4x6x8: 960 sites per parity), fewer RHS than warps, one and two RHS per warp."""
    m = 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    bs = list(I.make_sources(dims, nrhs, first_seed=2))
    rig = H.Rig(dims, U, precs=sorted({"double", inner}))
    rc, infos, x, y = _mrhs(H, rig, bs, m, inner, rb=-1)
    assert rc == Q.QCD_OK, infos
    for r in range(nrhs):
        assert infos[r]["converged"] and infos[r]["true_rel_residual"] <= 1e-10
        assert S.true_residual(U, x[r], bs[r], dims, m) <= 1.01e-10
        assert H.rel(y[r], S.dslash_parity(U, x[r], dims, 1)) <= 1e-12
    for r in (0, nrhs - 1):
        ref = S.cg_solve(U, bs[r], dims, m, tol=1e-12, max_iter=5000)
        assert H.rel(x[r], ref["x"]) <= _kappa(m) * 1e-10


def test_mrhs_fp64_agrees_with_single_rhs_solves(H):
    """The multi-RHS FP64 solve follows the single-RHS recursion (the single-RHS operator splits a
    small lattice's hops over lane pairs, so the rounding order differs slightly)."""
    dims, m = (6, 6, 6, 6), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    bs = list(I.make_sources(dims, 4, first_seed=2))
    rig = H.Rig(dims, U, precs=["double"])
    for rb in (1, 2, 4):
        rc, infos, x, _ = _mrhs(H, rig, bs, m, "double", rb=rb)
        assert rc == Q.QCD_OK
        for r in range(4):
            _, info1, x1, _ = rig.cg(bs[r], m)
            assert abs(info1["iterations"] - infos[r]["iterations"]) <= 1
            assert H.rel(x[r], x1) <= 1e-9, (rb, r)


def test_mrhs_results_agree_across_rhs_blocks(H):
    """Every register block solves the same systems; the grid (and so the reduction order) differs
    with the block, so the solutions agree to the solve's own accuracy (kappa * tol), and a
    repeated run with the same block is bit-identical."""
    dims, m = (4, 4, 6, 8), 0.05
    U = I.make_links(dims, kind="haar", seed=3)
    bs = list(I.make_sources(dims, 5, first_seed=7))
    rig = H.Rig(dims, U, precs=["double", "single12"])
    outs = [_mrhs(H, rig, bs, m, "single12", rb=rb)[2] for rb in (1, 2, 4, 8, 16, -1)]
    for o in outs[1:]:
        for r in range(5):
            assert H.rel(o[r], outs[0][r]) <= _kappa(m) * 2e-10
    again = _mrhs(H, rig, bs, m, "single12", rb=4)[2]
    assert np.array_equal(again, outs[2])


def test_mrhs_status_per_rhs(H):
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="haar", seed=1)
    bs = list(I.make_sources(dims, 3, first_seed=2))
    bs[1] = bs[1].copy()
    bs[1][5, 2] = np.nan
    bs[2] = np.zeros_like(bs[2])
    rig = H.Rig(dims, U, precs=["double", "single12"])
    for inner in ("double", "single12"):
        rc, infos, x, _ = _mrhs(H, rig, bs, 0.1, inner)
        assert rc == Q.QCD_ERR_BREAKDOWN
        assert infos[0]["converged"] and infos[0]["true_rel_residual"] <= 1e-10
        assert infos[1]["status"] == Q.QCD_ERR_BREAKDOWN
        assert infos[2]["converged"] and infos[2]["iterations"] == 0 and not np.any(x[2])
    rc, infos, _, _ = _mrhs(H, rig, bs[:1], 0.1, "double", max_iter=5)
    assert rc == Q.QCD_ERR_NOT_CONVERGED and infos[0]["iterations"] == 5


def test_full_size_24_4_sixteen_rhs(H):
    """24^4, 16 Gaussian right-hand sides, m = 0.05, FP32 recon-12 inner with FP64 reliable updates."""
    dims, m = (24, 24, 24, 24), 0.05
    U = I.make_links(dims, kind="haar", seed=1)
    bs = list(I.make_sources(dims, 16, first_seed=2))
    rig = H.Rig(dims, U, precs=["double", "single12"])
    rc, infos, x, y = _mrhs(H, rig, bs, m, "single12", want_y=False)
    assert rc == Q.QCD_OK, [i["status"] for i in infos]
    rng = np.random.default_rng(1)
    V = S.volume(dims)
    cand = rng.choice(V, 3000, replace=False)
    sites = cand[S.parity_of_sites(dims, cand) == 0][:800]
    for r in (0, 7, 15):
        assert infos[r]["true_rel_residual"] <= 1e-10
        res = bs[r][sites] - S.mdagm_sites(U, x[r], dims, m, sites)
        assert np.linalg.norm(res) / np.linalg.norm(bs[r][sites]) <= 3e-10


# ---------------------------------------------------------------- persistent multi-lattice solve


class Batch:
    def __init__(self, H, specs, inner):
        import torch
        self.torch = torch
        self.specs = specs
        self.inner = inner
        self.rigs, self.U, self.b = [], [], []
        for dims, m, ls, ss in specs:
            U = I.make_links(dims, kind="haar", seed=ls)
            self.U.append(U)
            self.b.append(I.make_source(dims, seed=ss))
            self.rigs.append(H.Rig(dims, U, precs=sorted({"double", inner})))
        self.opts = Q.qcd_solver_opts_default()
        self.opts.prec_inner, self.opts.recon_inner = H.PRECS[inner]
        self.lats = [r.h for r in self.rigs]
        nbytes = Q.qcd_workspace_bytes_batched(self.lats, self.opts)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.bd = [H.dev(b) for b in self.b]
        self.H = H

    def solve(self, cluster=0, block=0, tol=1e-10, max_iter=20000, use_graph=1):
        torch = self.torch
        self.opts.cluster_size, self.opts.block_size, self.opts.use_graph = cluster, block, use_graph
        xs = [torch.zeros_like(b) for b in self.bd]
        ys = [torch.zeros_like(b) for b in self.bd]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        rc, infos = Q.qcd_cg_solve_batched(self.lats, xs, self.bd, ys, [sp[1] for sp in self.specs], tol, max_iter,
                                           self.opts, self.ws, stream=s)
        s.synchronize()
        return rc, infos, [self.H.host(t) for t in xs], [self.H.host(t) for t in ys]


SMALL_BATCH = [((4, 4, 4, 4), 0.3, 11, 21), ((6, 6, 6, 6), 0.05, 12, 22), ((2, 4, 6, 8), 0.1, 13, 23),
               ((8, 8, 8, 8), 0.02, 14, 24), ((4, 4, 4, 8), 0.5, 15, 25), ((8, 8, 8, 16), 0.2, 16, 26),
               ((6, 4, 2, 4), 0.07, 17, 27)]


@pytest.mark.parametrize("inner", ["double", "single12", "half12", "df64"])
def test_batched_matches_oracle(H, inner):
    B = Batch(H, SMALL_BATCH, inner)
    refs = [S.cg_solve(B.U[i], B.b[i], sp[0], sp[1], tol=1e-12, max_iter=20000) for i, sp in enumerate(SMALL_BATCH)]
    for cluster in (1, 2, 4, 8, 16):
        rc, infos, xs, ys = B.solve(cluster=cluster, block=128 if cluster == 16 else 256)
        assert rc == Q.QCD_OK, (cluster, [i["status"] for i in infos])
        for i, (dims, m, _, _) in enumerate(SMALL_BATCH):
            assert infos[i]["true_rel_residual"] <= 1e-10
            assert S.true_residual(B.U[i], xs[i], B.b[i], dims, m) <= 1.01e-10, (cluster, i)
            assert H.rel(xs[i], refs[i]["x"]) <= _kappa(m) * 1e-10
            assert H.rel(ys[i], S.dslash_parity(B.U[i], xs[i], dims, 1)) <= 1e-12
            if inner != "double":
                assert infos[i]["reliable_updates"] >= 1


def test_batched_fp64_agrees_with_single_solves(H):
    B = Batch(H, SMALL_BATCH[:4], "double")
    rc, infos, xs, _ = B.solve(cluster=2, use_graph=0)
    assert rc == Q.QCD_OK
    for i, (dims, m, _, _) in enumerate(SMALL_BATCH[:4]):
        _, info1, x1, _ = B.rigs[i].cg(B.b[i], m)
        assert abs(info1["iterations"] - infos[i]["iterations"]) <= 1
        assert H.rel(xs[i], x1) <= 1e-9


def test_batched_status_codes(H):
    specs = SMALL_BATCH[:3]
    B = Batch(H, specs, "single12")
    B.b[1] = B.b[1].copy()
    B.b[1][0, 0] = np.nan  # site 0 is even: the solve reads it
    B.bd[1] = H.dev(B.b[1])
    rc, infos, xs, _ = B.solve(cluster=2)
    assert rc == Q.QCD_ERR_BREAKDOWN
    assert infos[1]["status"] == Q.QCD_ERR_BREAKDOWN
    assert infos[0]["converged"] and infos[2]["converged"]
    rc, infos, _, _ = B.solve(cluster=2, max_iter=4)
    assert rc in (Q.QCD_ERR_NOT_CONVERGED, Q.QCD_ERR_BREAKDOWN)
    assert infos[0]["status"] == Q.QCD_ERR_NOT_CONVERGED and infos[0]["iterations"] == 4


def test_full_batch_of_64_uneven_lattices(H):
    """64 lattices drawn from {4^4, 6^4, 8^4, 8^3x16}, m in [0.02, 0.5], one persistent launch."""
    specs = I.make_lattice_batch(64, seed=4)
    B = Batch(H, specs, "single12")
    rc, infos, xs, ys = B.solve()
    assert rc == Q.QCD_OK, [i["status"] for i in infos]
    for i, (dims, m, _, _) in enumerate(specs):
        assert infos[i]["true_rel_residual"] <= 1e-10
        assert S.true_residual(B.U[i], xs[i], B.b[i], dims, m) <= 1.01e-10, i


def test_autotuners_pick_valid_shapes_and_cache_them(H):
    dims, m = (8, 8, 8, 8), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    rig = H.Rig(dims, U, precs=["double", "single12"])
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = Q.QCD_PREC_SINGLE, 12
    bs = I.make_sources(dims, 8, first_seed=2)
    bd = H.dev(bs)
    import torch
    x = torch.zeros_like(bd)
    ws = rig.lat.workspace(opts, 8)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        rb = Q.qcd_tune_mrhs(rig.h, 8, x, bd, m, opts, ws, cache_path=path)
        assert rb in (-1, 1, 2, 4, 8, 16)  # -1: the shared-link kernel, a candidate from 2 RHS on
        B = Batch(H, SMALL_BATCH[:4], "single12")
        c, blk = Q.qcd_tune_batched(B.lats, [torch.zeros_like(b) for b in B.bd], B.bd, [s[1] for s in B.specs],
                                    1e-10, 20000, B.opts, B.ws, cache_path=path)
        assert c in (1, 2, 4, 8, 16) and blk in (128, 256)
        lines = open(path).read().split("\n")
        assert any(ln.startswith("mrhs|") and ln.split()[1] == str(rb) for ln in lines)
        assert any(ln.startswith("batched|") and ln.split()[1:3] == [str(c), str(blk)] for ln in lines)
        Q.qcd_tune_load(path)
        # the tuned shapes are used when the options leave them at 0
        rc, infos, _, _ = B.solve(cluster=0, block=0)
        assert rc == Q.QCD_OK
