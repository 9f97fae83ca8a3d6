"""The C-ABI library loads, exports every symbol include/qcd.h declares, and validates arguments
on the host (no GPU needed: these calls fail before any device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"QCD_API\s+[\w\s\*]+?\b(qcd_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_symbols()
    for must in ["qcd_lattice_create", "qcd_load_links", "qcd_dslash", "qcd_mdagm", "qcd_cg_solve"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1311_2719_gb300 import qcd as Q
    lib = ctypes.CDLL(Q.LIB_PATH)
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps exactly the declared surface
    assert set(Q.SIGNATURES) == set(_declared_symbols())


def test_lattice_validation_and_sizes():
    from paper_1311_2719_gb300 import qcd as Q
    for bad in [(3, 4, 4, 4), (4, 0, 4, 4), (4, 4, 4, 1), (4, 4, -2, 4)]:
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_lattice_create(*bad)
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
    h = Q.qcd_lattice_create(4, 4, 4, 8)
    try:
        Vh = 4 * 4 * 4 * 8 // 2
        assert Q.qcd_field_bytes(h, Q.QCD_PREC_DOUBLE) == Vh * 48
        assert Q.qcd_field_bytes(h, Q.QCD_PREC_SINGLE) == Vh * 24
        assert Q.qcd_field_bytes(h, Q.QCD_PREC_HALF) == Vh * 16
        assert Q.qcd_field_bytes(h, 7) == 0
        assert Q.qcd_links_bytes(h, Q.QCD_PREC_DOUBLE, 18) == 2 * Vh * 4 * 144
        assert Q.qcd_links_bytes(h, Q.QCD_PREC_SINGLE, 18) == 2 * Vh * 4 * 72
        assert Q.qcd_links_bytes(h, Q.QCD_PREC_SINGLE, 12) == 2 * Vh * 4 * 48
        assert Q.qcd_links_bytes(h, Q.QCD_PREC_HALF, 12) == 2 * Vh * 4 * 24
        assert Q.qcd_links_bytes(h, Q.QCD_PREC_DOUBLE, 12) == 0
        o = Q.qcd_solver_opts_default()
        assert (o.prec_inner, o.recon_inner, o.reliable_interval) == (0, 18, 100)
        assert Q.qcd_workspace_bytes(h, o) > 4 * Vh * 48
        assert Q.qcd_lattice_set_tbc(h, 1) is None
        with pytest.raises(Q.QcdError):
            Q.qcd_lattice_set_tbc(h, 0)
    finally:
        Q.qcd_lattice_destroy(h)


def test_calls_reject_bad_arguments_before_device_work():
    from paper_1311_2719_gb300 import qcd as Q
    h = Q.qcd_lattice_create(4, 4, 4, 4)
    try:
        fake = 1 << 20  # an aligned address that is never dereferenced: validation fails first
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_dslash(h, fake, fake, 0, Q.QCD_PREC_DOUBLE)  # aliasing
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_dslash(h, fake, fake + 256, 2, Q.QCD_PREC_DOUBLE)  # bad parity
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_dslash(h, fake, fake + 256, 0, Q.QCD_PREC_DOUBLE)  # no links loaded
        assert e.value.status == Q.QCD_ERR_NO_LINKS
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_dslash(h, fake + 8, fake + 256, 0, Q.QCD_PREC_DOUBLE)  # misaligned
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_dslash_mrhs(h, fake, fake + 256, 17, 0, Q.QCD_PREC_SINGLE)
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_mdagm(h, fake, fake + 256, -0.1, Q.QCD_PREC_DOUBLE, fake + 512)
        assert e.value.status == Q.QCD_ERR_INVALID_ARG
        with pytest.raises(Q.QcdError) as e:
            Q.qcd_load_links(h, fake, fake + 256, Q.QCD_PREC_DOUBLE, 12)
        assert e.value.status == Q.QCD_ERR_UNSUPPORTED
        o = Q.qcd_solver_opts_default()
        for mass, tol, it in [(0.0, 1e-10, 10), (0.1, 0.0, 10), (0.1, 1e-10, 0), (float("nan"), 1e-10, 10)]:
            rc, info = Q.qcd_cg_solve(h, fake, fake + 256, mass, tol, it, o, fake + 512, raise_on=())
            assert rc == Q.QCD_ERR_INVALID_ARG and info["status"] == rc
        rc, _ = Q.qcd_cg_solve(h, fake, fake + 256, 0.1, 1e-10, 10, o, fake + 512, raise_on=())
        assert rc == Q.QCD_ERR_NO_LINKS
        # batched launch shapes: 0 (tuned) or a supported cluster / block size
        for cs, bs in [(3, 0), (-4, 0), (32, 0), (0, 100), (0, 16), (0, 512), (0, -32)]:
            ob = Q.qcd_solver_opts_default()
            ob.cluster_size, ob.block_size = cs, bs
            rc, _ = Q.qcd_cg_solve_batched([h], [fake], [fake + 256], None, [0.1], 1e-10, 10, ob, fake + 512,
                                           raise_on=())
            assert rc == Q.QCD_ERR_INVALID_ARG, (cs, bs)
        rc, _ = Q.qcd_cg_solve_batched([h], [fake], [fake + 256], None, [0.1], 1e-10, 10,
                                       Q.qcd_solver_opts_default(), fake + 512, raise_on=())
        assert rc == Q.QCD_ERR_NO_LINKS
    finally:
        Q.qcd_lattice_destroy(h)


def test_solver_opts_layout_matches_the_library():
    """The ctypes mirror of qcd_solver_opts covers every field the library writes: the default
    fill reaches the last field (prec_outer) and nothing past the struct."""
    import ctypes
    from paper_1311_2719_gb300 import qcd as Q
    n = ctypes.sizeof(Q.qcd_solver_opts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    o = Q.qcd_solver_opts.from_buffer(buf)
    o.prec_outer = 99
    Q._lib.qcd_solver_opts_default(ctypes.byref(o))
    assert o.prec_outer == Q.QCD_PREC_DOUBLE and o.staged == 0 and o.wait_cycles == 0
    assert bytes(buf[n:]) == b"\xab" * 64


def test_wilson_byte_counts():
    from paper_1311_2719_gb300 import qcd as Q
    h = Q.qcd_lattice_create(4, 2, 6, 8)
    try:
        V = 4 * 2 * 6 * 8
        assert Q.qcd_wilson_field_bytes(h, Q.QCD_PREC_DOUBLE) == V * 12 * 16
        assert Q.qcd_wilson_field_bytes(h, Q.QCD_PREC_SINGLE) == V * 12 * 8
        assert Q.qcd_wilson_field_bytes(h, Q.QCD_PREC_DF64) == V * 12 * 16
        assert Q.qcd_wilson_field_bytes(h, Q.QCD_PREC_HALF) == 0
        assert Q.qcd_wilson_links_bytes(h, Q.QCD_PREC_DOUBLE) == V * 4 * 9 * 16
        assert Q.qcd_wilson_links_bytes(h, Q.QCD_PREC_DF64) == V * 4 * 9 * 16
        assert Q.qcd_wilson_links_bytes(h, Q.QCD_PREC_SINGLE) == V * 4 * 9 * 8
        o = Q.qcd_solver_opts_default()
        o.prec_inner, o.prec_outer = Q.QCD_PREC_SINGLE, Q.QCD_PREC_DF64
        assert Q.qcd_wilson_workspace_bytes(h, o, 2) > 0
        o.prec_inner = Q.QCD_PREC_DOUBLE
        assert Q.qcd_wilson_workspace_bytes(h, o, 2) == 0
    finally:
        Q.qcd_lattice_destroy(h)


def test_tune_cache_loader_skips_shapes_the_solvers_reject(tmp_path):
    """qcd_tune_load parses its text cache on the host: a missing file is not an error, malformed
    or unsupported lines are skipped, a NULL path is rejected."""
    from paper_1311_2719_gb300 import qcd as Q
    Q.qcd_tune_load(str(tmp_path / "absent.txt"))
    p = tmp_path / "tune.txt"
    p.write_text("mrhs|X|4x4x4x4|p1|r12|n8 3 100\n"        # RHS block 3: not a shape
                 "mrhs|X|4x4x4x4|p1|r12|n8 -1 100\n"       # the shared-link kernel
                 "batched|X|n4|v1024|p1|r12 0 128 5\n"      # cluster 0
                 "batched|X|n4|v1024|p1|r12 4 100 5\n"      # block not a multiple of 32
                 "garbage\n\n"
                 "batched|X|n4|v1024|p1|r12 4 128\n")
    Q.qcd_tune_load(str(p))
    with pytest.raises(Q.QcdError) as e:
        Q._check(Q._lib.qcd_tune_load(None), "qcd_tune_load")
    assert e.value.status == Q.QCD_ERR_INVALID_ARG
