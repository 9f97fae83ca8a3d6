"""GPU even-odd CG vs the FP64 oracle (solution, opposite-parity image, residuals, status codes)."""
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


def _kappa_bound(m):
    # |D| <= 4 so the spectrum of A lies in [m^2, m^2 + 16]
    return (m * m + 16.0) / (m * m)


@pytest.mark.parametrize("dims,kind,m", [((4, 4, 4, 4), "haar", 0.1), ((2, 4, 6, 8), "haar", 0.1),
                                         ((6, 6, 6, 6), "near_identity", 0.05), ((8, 8, 8, 8), "haar", 0.1)])
def test_fp64_cg_matches_oracle(H, dims, kind, m):
    U = I.make_links(dims, kind=kind, seed=1)
    b = I.make_source(dims, seed=2)
    ref = S.cg_solve(U, b, dims, m, tol=1e-10, max_iter=5000)
    rig = H.Rig(dims, U, precs=["double"])
    rc, info, x, y = rig.cg(b, m, tol=1e-10)
    assert rc == Q.QCD_OK and info["converged"] == 1
    assert info["true_rel_residual"] <= 1e-10
    # an independent FP64 residual of the GPU solution, computed by the oracle
    assert S.true_residual(U, x, b, dims, m) <= 1.01e-10
    # same recursion in the same order: iteration counts agree closely, solutions to ~kappa * tol
    assert abs(info["iterations"] - ref["iterations"]) <= 2
    err = H.rel(x, ref["x"])
    assert err <= _kappa_bound(m) * 1e-10 and err <= 1e-8, err
    assert H.rel(y, ref["y"]) <= 1e-8
    # y is D_oe x exactly as the half-lattice operator defines it
    assert H.rel(y, S.dslash_parity(U, x, dims, 1)) <= 1e-12
    assert np.all(x[S.parity(dims) == 1] == 0) and np.all(y[S.parity(dims) == 0] == 0)


def test_free_field_converges_in_four_iterations(H):
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="unit")
    rig = H.Rig(dims, U, precs=["double"])
    rc, info, x, _ = rig.cg(I.make_source(dims, seed=2), 0.1, tol=1e-10, check_interval=1)
    assert rc == Q.QCD_OK and info["iterations"] <= 5


def test_graph_replay_equals_eager_bitwise(H):
    dims = (6, 6, 6, 6)
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "single12"])
    for inner in ("double", "single12"):
        _, i1, x1, y1 = rig.cg(b, 0.1, use_graph=1, check_interval=8, inner=inner)
        _, i2, x2, y2 = rig.cg(b, 0.1, use_graph=0, check_interval=8, inner=inner)
        assert i1["iterations"] == i2["iterations"]
        assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
        # deterministic reductions: a second run is bit-identical too
        _, _, x3, _ = rig.cg(b, 0.1, use_graph=1, check_interval=8, inner=inner)
        assert np.array_equal(x1, x3)


@pytest.mark.parametrize("inner", ["single18", "single12", "half12", "df64"])
@pytest.mark.parametrize("dims,m", [((8, 8, 8, 8), 0.1), ((6, 6, 6, 6), 0.02)])
def test_mixed_precision_cg_reaches_fp64_residual(H, inner, dims, m):
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    ref = S.cg_solve(U, b, dims, m, tol=1e-12, max_iter=20000)
    rig = H.Rig(dims, U, precs=["double", inner])
    rc, info, x, y = rig.cg(b, m, tol=1e-10, inner=inner)
    assert rc == Q.QCD_OK, info
    assert info["true_rel_residual"] <= 1e-10 and info["reliable_updates"] >= 1
    assert S.true_residual(U, x, b, dims, m) <= 1.01e-10
    assert H.rel(x, ref["x"]) <= _kappa_bound(m) * 1e-10
    assert H.rel(y, S.dslash_parity(U, x, dims, 1)) <= 1e-12


def test_status_codes(H):
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="haar", seed=1)
    rig = H.Rig(dims, U, precs=["double", "single12"])
    b = I.make_source(dims, seed=2)
    # max_iter exhausted
    rc, info, _, _ = rig.cg(b, 0.1, max_iter=3, check_interval=1)
    assert rc == Q.QCD_ERR_NOT_CONVERGED and info["iterations"] == 3 and not info["converged"]
    # injected breakdown: a NaN in the source
    bn = b.copy()
    bn[0, 1] = np.nan
    for inner in ("double", "single12"):
        rc, info, _, _ = rig.cg(bn, 0.1, inner=inner)
        assert rc == Q.QCD_ERR_BREAKDOWN
    # zero source: x = 0 exactly, converged without iterating
    rc, info, x, y = rig.cg(np.zeros_like(b), 0.1)
    assert rc == Q.QCD_OK and info["iterations"] == 0 and not np.any(x) and not np.any(y)


@pytest.mark.parametrize("kind,m", [("near_identity", 0.5), ("haar", 0.5), ("haar", 0.1), ("haar", 0.02),
                                    ("near_identity", 0.02)])
def test_full_size_16_4_fp64(H, kind, m):
    """16^4, FP64 CG to 1e-10 at every mass of the workload; oracle solution where it is quick."""
    dims = (16, 16, 16, 16)
    U = I.make_links(dims, kind=kind, seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double"])
    rc, info, x, y = rig.cg(b, m, tol=1e-10)
    assert rc == Q.QCD_OK and info["true_rel_residual"] <= 1e-10
    assert S.true_residual(U, x, b, dims, m) <= 1.01e-10
    if m >= 0.5:
        ref = S.cg_solve(U, b, dims, m, tol=1e-10, max_iter=1000)
        assert H.rel(x, ref["x"]) <= 1e-8


@pytest.mark.parametrize("inner", ["single12", "half12"])
def test_full_size_32_4_mixed(H, inner):
    """32^4, m = 0.01: mixed CG reaches a true FP64 residual of 1e-10 (sampled oracle residual)."""
    dims = (32, 32, 32, 32)
    m = 0.01
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", inner])
    rc, info, x, y = rig.cg(b, m, tol=1e-10, inner=inner, max_iter=40000)
    assert rc == Q.QCD_OK, info
    assert info["true_rel_residual"] <= 1e-10
    # sampled FP64 residual by the oracle: |b - A x| at 2000 even sites relative to |b| there
    rng = np.random.default_rng(0)
    V = S.volume(dims)
    cand = rng.choice(V, 6000, replace=False)
    sites = cand[S.parity_of_sites(dims, cand) == 0][:2000]
    r = b[sites] - S.mdagm_sites(U, x, dims, m, sites)
    assert np.linalg.norm(r) / np.linalg.norm(b[sites]) <= 3e-10


def test_df64_cg_full_size_16_4(H):
    """16^4, m = 0.1: the df64 recursion (FP32 pipes, 48-bit significand) with FP64 confirmation."""
    dims, m = (16, 16, 16, 16), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "df64"])
    rc, info, x, y = rig.cg(b, m, tol=1e-10, inner="df64")
    assert rc == Q.QCD_OK and info["true_rel_residual"] <= 1e-10
    assert S.true_residual(U, x, b, dims, m) <= 1.01e-10
    _, info64, x64, _ = rig.cg(b, m, tol=1e-10)
    # same recursion up to rounding: iteration counts within a few, solutions to ~kappa * tol
    assert abs(info["iterations"] - info64["iterations"]) <= 5
    assert H.rel(x, x64) <= 1e-8


def _solve_full(H, rig, b, m, tol=1e-10, inner="double"):
    import torch
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = H.PRECS[inner]
    ws = torch.empty(Q.qcd_workspace_bytes_full(rig.h, opts), dtype=torch.uint8, device="cuda")
    bd = H.dev(b)
    x = torch.zeros_like(bd)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rc, info = Q.qcd_solve_full(rig.h, x, bd, m, tol, 20000, opts, ws, stream=s)
    s.synchronize()
    return rc, info, H.host(x)


@pytest.mark.parametrize("inner", ["double", "single12", "half12", "df64"])
@pytest.mark.parametrize("dims,m", [((2, 4, 6, 8), 0.1), ((6, 6, 6, 6), 0.05), ((4, 4, 4, 8), 0.5)])
def test_full_system_solve_matches_oracle(H, inner, dims, m):
    """M x = b on both parities (M = m + D): GPU even-odd reduction vs the oracle's full-lattice CG."""
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=sorted({"double", inner}))
    rc, info, x = _solve_full(H, rig, b, m, 1e-10, inner)
    assert rc == Q.QCD_OK, info
    assert info["true_rel_residual"] <= 1e-10
    res = b - S.apply_m(U, x, dims, m)
    assert np.linalg.norm(res) / np.linalg.norm(b) <= 1.01e-10
    ref = S.solve_full(U, b, dims, m, tol=1e-13, max_iter=20000)
    assert H.rel(x, ref["x"]) <= (1.0 + 4.0 / m) * 1e-10 * 10


def test_full_system_solve_16_4(H):
    dims, m = (16, 16, 16, 16), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "df64"])
    for inner in ("double", "df64"):
        rc, info, x = _solve_full(H, rig, b, m, 1e-10, inner)
        assert rc == Q.QCD_OK and info["true_rel_residual"] <= 1e-10
        res = b - S.apply_m(U, x, dims, m)
        assert np.linalg.norm(res) / np.linalg.norm(b) <= 1.01e-10


@pytest.mark.parametrize("dims,m", [((8, 8, 8, 8), 0.1), ((2, 4, 6, 8), 0.1), ((10, 4, 6, 8), 0.05), ((6, 6, 6, 6), 0.02),
                                    ((16, 16, 16, 16), 0.1)])
def test_staged_operator_cg_matches_oracle_and_direct(H, dims, m):
    """The FP32 recon-12 CG with the operator's inputs staged in shared memory by bulk copies: same
    solution as the oracle, graph == eager, and the same recursion as the direct-load kernel up to
    rounding (ragged last tiles, runs clamped at both ends of the index range, wrapped neighbours)."""
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "single12"])
    rc, info, x, y = rig.cg(b, m, inner="single12", staged=1)
    assert rc == Q.QCD_OK, info
    assert info["true_rel_residual"] <= 1e-10
    assert S.true_residual(U, x, b, dims, m) <= 1.01e-10
    ref = S.cg_solve(U, b, dims, m, tol=1e-12, max_iter=20000)
    assert H.rel(x, ref["x"]) <= _kappa_bound(m) * 1e-10
    rc_e, info_e, x_e, _ = rig.cg(b, m, inner="single12", staged=1, use_graph=0)
    assert rc_e == Q.QCD_OK and info_e["iterations"] == info["iterations"] and np.array_equal(x, x_e)
    rc_d, info_d, x_d, _ = rig.cg(b, m, inner="single12", staged=0)
    assert rc_d == Q.QCD_OK and abs(info_d["iterations"] - info["iterations"]) <= 2
    assert H.rel(x, x_d) <= _kappa_bound(m) * 2e-10


def test_staged_operator_wait_limit_reports_timeout(H):
    """Failure detection without a GPU fault: a wait limit of one clock cycle makes the staged
    operator's first wait on its bulk copies give up; the kernel records the fault, lets its copies
    land, and the solve returns QCD_ERR_TIMEOUT. A default solve on the same buffers then succeeds."""
    import torch
    dims, m = (8, 8, 8, 8), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=["double", "single12"])
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = PRECS_SINGLE12
    opts.staged, opts.wait_cycles = 1, 1
    ws = rig.lat.workspace(opts)
    bd = H.dev(b)
    x, y = torch.zeros_like(bd), torch.zeros_like(bd)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rc, info = Q.qcd_cg_solve(rig.h, x, bd, m, 1e-10, 1000, opts, ws, y, stream=s, raise_on=())
    s.synchronize()
    assert rc == Q.QCD_ERR_TIMEOUT and info["status"] == Q.QCD_ERR_TIMEOUT
    opts.wait_cycles = 0
    rc, info = Q.qcd_cg_solve(rig.h, x, bd, m, 1e-10, 1000, opts, ws, y, stream=s, raise_on=())
    s.synchronize()
    assert rc == Q.QCD_OK and info["true_rel_residual"] <= 1e-10


PRECS_SINGLE12 = (Q.QCD_PREC_SINGLE, 12)
