"""GPU fermion force vs the FP64 force oracle, through the C-ABI."""
import numpy as np
import pytest

from oracle import force as F
from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I
from paper_1311_2719_gb300 import qcd as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from tests import gpu_helpers
    return gpu_helpers


def _gpu_force(H, lat, U, x, y):
    import torch
    f = torch.zeros((lat.V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    Q.qcd_fermion_force(lat.handle, f, H.dev(U), H.dev(x), H.dev(y))
    torch.cuda.synchronize()
    return H.host(f)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 6, 8), (6, 4, 2, 4), (4, 6, 4, 10)])
@pytest.mark.parametrize("tbc", [-1, 1])
def test_force_matches_oracle(H, dims, tbc):
    U = I.make_links(dims, kind="haar", seed=1)
    x, y = I.make_source(dims, seed=2), I.make_source(dims, seed=3)  # the kernel reads x even, y odd only
    lat = Q.Lattice(dims, tbc=tbc)
    got = _gpu_force(H, lat, U, x, y)
    want = F.fermion_force(U, x, y, dims, tbc=float(tbc))
    assert H.rel(got, want) <= 1e-13


def test_force_ignores_other_parity(H):
    dims = (4, 4, 2, 6)
    U = I.make_links(dims, kind="haar", seed=1)
    x, y = I.make_source(dims, seed=2), I.make_source(dims, seed=3)
    par = S.parity(dims)
    lat = Q.Lattice(dims)
    a = _gpu_force(H, lat, U, x, y)
    b = _gpu_force(H, lat, U, np.where((par == 0)[:, None], x, 0.0), np.where((par == 1)[:, None], y, 0.0))
    assert np.array_equal(a, b)


def test_force_from_gpu_cg_solution(H):
    """x and y from qcd_cg_solve feed the force; compared with the force of the oracle's own CG."""
    import torch
    dims, mass = (4, 4, 4, 4), 0.1
    U = I.make_links(dims, kind="haar", seed=1)
    phi = I.make_source(dims, seed=2)
    rig = H.Rig(dims, U, precs=("double",))
    opts = Q.qcd_solver_opts_default()
    ws = rig.lat.workspace(opts)
    b = H.dev(phi)
    x, y = torch.zeros_like(b), torch.zeros_like(b)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rc, info = Q.qcd_cg_solve(rig.h, x, b, mass, 1e-12, 10000, opts, ws, y, stream=s)
    s.synchronize()
    assert rc == Q.QCD_OK
    got = _gpu_force(H, rig.lat, U, H.host(x), H.host(y))
    ref = S.cg_solve(U, phi, dims, mass, 1e-13, 10000)
    want = F.fermion_force(U, ref["x"], S.dslash_parity(U, ref["x"], dims, 1), dims)
    assert H.rel(got, want) <= 1e-9


def test_force_full_size_32_sampled(H):
    dims = (32, 32, 32, 32)
    U = I.make_links(dims, kind="haar", seed=1)
    x, y = I.make_source(dims, seed=2), I.make_source(dims, seed=3)
    lat = Q.Lattice(dims)
    got = _gpu_force(H, lat, U, x, y)
    V = S.volume(dims)
    rng = np.random.default_rng(11)
    sites = np.concatenate([rng.choice(V, 3000, replace=False), [0, V - 1]])
    mus = np.concatenate([rng.integers(0, 4, 3000), [3, 3]])
    want = F.fermion_force_links(U, x, y, dims, sites, mus)
    assert H.rel(got[sites, mus], want) <= 1e-13
    # every force matrix traceless Hermitian
    assert np.max(np.abs(got - np.conj(np.swapaxes(got, -1, -2)))) <= 1e-12
    assert np.max(np.abs(np.trace(got, axis1=-2, axis2=-1))) <= 1e-12


def test_force_argument_checks(H):
    import torch
    dims = (2, 2, 2, 2)
    lat = Q.Lattice(dims)
    U = H.dev(I.make_links(dims, kind="unit"))
    x = H.dev(I.make_source(dims, seed=2))
    f = torch.zeros((lat.V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(Q.QcdError):
        Q.qcd_fermion_force(lat.handle, U, U, x, x)
    with pytest.raises(Q.QcdError):
        Q.qcd_fermion_force(lat.handle, f, None, x, x)
