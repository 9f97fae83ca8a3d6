"""The allocation-free operator entry point (qcd_mdagm_noalloc) agrees with qcd_mdagm.

qcd_mdagm_noalloc serves callers that cannot allocate device memory (their device arrays come
from data directives, or another framework's pool owns every byte of the GPU): it keeps its
intermediate odd-parity field in a library-owned device array. It launches the same kernels as
qcd_mdagm on the same inputs, so the two results must be bit-identical; each is also checked
against the FP64 oracle at the operator tolerance of its precision. This file is named so that
pytest collects it last; it must pass both on its own in a fresh process and after every other
test.
"""
import numpy as np
import pytest

from oracle import staggered as S
from paper_1311_2719_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"double": 1e-12, "single12": 1e-5, "half12": 5e-3, "df64": 1e-12}


def _both(rig, name, x, mass, stream):
    """(qcd_mdagm with caller scratch, qcd_mdagm_noalloc) on the same packed input, both on `stream`."""
    from paper_1311_2719_gb300 import qcd as Q
    from tests import gpu_helpers as H

    prec = H.PRECS[name][0]
    cur = rig.torch.cuda.current_stream()
    fin = rig.pack(H.dev(x), Q.QCD_EVEN, prec)
    want_f, tmp, got_f = rig.lat.field(prec), rig.lat.field(prec), rig.lat.field(prec)
    stream.wait_stream(cur)
    Q.qcd_mdagm(rig.h, want_f, fin, mass, prec, tmp, stream=stream)
    Q.qcd_mdagm_noalloc(rig.h, got_f, fin, mass, prec, stream=stream)
    cur.wait_stream(stream)
    want = rig.unpack(want_f, Q.QCD_EVEN, prec)
    got = rig.unpack(got_f, Q.QCD_EVEN, prec)
    rig.torch.cuda.synchronize()
    return H.host(want), H.host(got)


@pytest.mark.parametrize("name", ["double", "single12", "half12", "df64"])
def test_noalloc_matches_caller_scratch_twice(name):
    import torch

    from tests import gpu_helpers as H

    dims = (8, 6, 4, 10)  # 960 sites per parity: several blocks and a ragged tail
    U = I.make_links(dims, kind="haar", seed=1)
    rig = H.Rig(dims, U, precs=[name])
    stream = torch.cuda.Stream()
    for call, (seed, mass) in enumerate([(3, 0.1), (4, 0.35)]):  # two calls in a row
        x = I.make_source(dims, seed=seed)
        want, got = _both(rig, name, x, mass, stream)
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, want), (name, call, H.rel(got, want))
        assert H.rel(got, S.mdagm(U, x, dims, mass)) <= TOL[name], (name, call)


def test_noalloc_across_lattices_and_precisions():
    """The shared array keeps the previous call's contents: a larger lattice at FP64, then a
    smaller one at FP16, then the larger one again at FP32, each bit-identical to qcd_mdagm."""
    import torch

    from tests import gpu_helpers as H

    stream = torch.cuda.Stream()
    big, small = (12, 12, 12, 16), (4, 6, 2, 8)
    rigs = {}
    for dims in (big, small):
        U = I.make_links(dims, kind="haar", seed=1)
        rigs[dims] = (H.Rig(dims, U, precs=["double", "single12", "half12"]), U)
    for dims, name, mass in [(big, "double", 0.2), (small, "half12", 0.1), (big, "single12", 0.05),
                             (small, "double", 0.3)]:
        rig, U = rigs[dims]
        x = I.make_source(dims, seed=5)
        want, got = _both(rig, name, x, mass, stream)
        assert np.array_equal(got, want), (dims, name)
        assert H.rel(got, S.mdagm(U, x, dims, mass)) <= TOL[name], (dims, name)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    from paper_1311_2719_gb300 import qcd as Q
    from tests import gpu_helpers as H

    dims = (32, 32, 32, 24)  # FP64 odd field of 393216 sites = 18.9 MB > 16 MiB
    rig = H.Rig(dims, I.make_links(dims, kind="unit"), precs=["double"])
    f_in = rig.lat.field(Q.QCD_PREC_DOUBLE)
    f_out = rig.lat.field(Q.QCD_PREC_DOUBLE)
    with pytest.raises(Q.QcdError) as e:
        Q.qcd_mdagm_noalloc(rig.h, f_out, f_in, 0.1, Q.QCD_PREC_DOUBLE)
    assert e.value.status == Q.QCD_ERR_INVALID_ARG
    assert "16777216" in str(e.value)
