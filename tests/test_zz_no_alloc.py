"""The allocation-free operator entry point (qcd_mdagm_noalloc) agrees with qcd_mdagm.

qcd_mdagm_noalloc serves callers that cannot allocate device memory (their device arrays come
from data directives or from another framework's pool): it keeps its intermediate field in a
library-owned device array. This file is named so that pytest collects it last; it must pass
both on its own in a fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_1311_2719_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"double": 1e-12, "single12": 1e-5, "half12": 5e-3}


@pytest.mark.parametrize("name", ["double", "single12", "half12"])
def test_noalloc_matches_caller_scratch_twice(name):
    from paper_1311_2719_gb300 import qcd as Q
    from tests import gpu_helpers as H

    dims = (8, 6, 4, 10)  # 960 sites per parity: several blocks and a ragged tail
    rig = H.Rig(dims, I.make_links(dims, kind="haar", seed=1), precs=[name])
    prec = H.PRECS[name][0]
    for call, (seed, mass) in enumerate([(3, 0.1), (4, 0.35)]):  # two calls in a row
        x = I.make_source(dims, seed=seed)
        fin = rig.pack(H.dev(x), Q.QCD_EVEN, prec)
        want_f = rig.lat.field(prec)
        tmp = rig.lat.field(prec)
        Q.qcd_mdagm(rig.h, want_f, fin, mass, prec, tmp)
        got_f = rig.lat.field(prec)
        Q.qcd_mdagm_noalloc(rig.h, got_f, fin, mass, prec)
        want = H.host(rig.unpack(want_f, Q.QCD_EVEN, prec))
        got = H.host(rig.unpack(got_f, Q.QCD_EVEN, prec))
        assert np.all(np.isfinite(got))
        assert H.rel(got, want) <= TOL[name], (name, call, H.rel(got, want))


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
