"""ctypes binding of libqcd.so (include/qcd.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no arithmetic of its
own; all work happens in the CUDA kernels of the library. Device buffers are passed as raw
addresses (an int, or any object with ``data_ptr()`` such as a torch tensor); streams as a
``cudaStream_t`` address (``torch.cuda.current_stream().cuda_stream``) or None.

If the shared library is missing this module raises at import time: there is no fallback.
The :class:`Lattice` helper at the end owns a handle plus torch-allocated packed links and
workspace, which is how the tests and the benchmark drive the library.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqcd.so")

QCD_OK = 0
QCD_ERR_INVALID_ARG = 1
QCD_ERR_CUDA = 2
QCD_ERR_NOT_CONVERGED = 3
QCD_ERR_BREAKDOWN = 4
QCD_ERR_TIMEOUT = 5
QCD_ERR_UNSUPPORTED = 6
QCD_ERR_NO_LINKS = 7

QCD_EVEN, QCD_ODD = 0, 1
QCD_PREC_DOUBLE, QCD_PREC_SINGLE, QCD_PREC_HALF, QCD_PREC_DF64 = 0, 1, 2, 3
PREC_NAMES = {"double": QCD_PREC_DOUBLE, "single": QCD_PREC_SINGLE, "half": QCD_PREC_HALF, "df64": QCD_PREC_DF64}


class QcdError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


class qcd_solver_opts(ctypes.Structure):
    _fields_ = [
        ("prec_inner", ctypes.c_int),
        ("recon_inner", ctypes.c_int),
        ("reliable_delta", ctypes.c_double),
        ("reliable_interval", ctypes.c_int),
        ("check_interval", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("rhs_block", ctypes.c_int),
        ("cluster_size", ctypes.c_int),
        ("block_size", ctypes.c_int),
        ("staged", ctypes.c_int),
        ("wait_cycles", ctypes.c_longlong),
        ("prec_outer", ctypes.c_int),
    ]


class qcd_solve_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("status", ctypes.c_int),
        ("true_rel_residual", ctypes.c_double),
        ("iterated_rel_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_int),
        ("dslash_launches", ctypes.c_int),
        ("dslash_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sz = ctypes.c_size_t

# name -> (restype, argtypes); this table is the whole exported surface of include/qcd.h.
SIGNATURES = {
    "qcd_status_string": (ctypes.c_char_p, [_i]),
    "qcd_last_error": (ctypes.c_char_p, []),
    "qcd_version": (ctypes.c_char_p, []),
    "qcd_lattice_create": (_i, [_i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "qcd_lattice_destroy": (_i, [_vp]),
    "qcd_lattice_set_tbc": (_i, [_vp, _i]),
    "qcd_lattice_device": (_i, [_vp]),
    "qcd_field_bytes": (_sz, [_vp, _i]),
    "qcd_links_bytes": (_sz, [_vp, _i, _i]),
    "qcd_workspace_bytes": (_sz, [_vp, ctypes.POINTER(qcd_solver_opts), _i]),
    "qcd_solver_opts_default": (None, [ctypes.POINTER(qcd_solver_opts)]),
    "qcd_load_links": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "qcd_pack_field": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "qcd_unpack_field": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "qcd_dslash": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "qcd_dslash_mrhs": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "qcd_mdagm": (_i, [_vp, _vp, _vp, _d, _i, _vp, _vp]),
    "qcd_mdagm_noalloc": (_i, [_vp, _vp, _vp, _d, _i, _vp]),
    "qcd_cg_solve": (_i, [_vp, _vp, _vp, _d, _d, _i, ctypes.POINTER(qcd_solver_opts), _vp, _vp,
                          ctypes.POINTER(qcd_solve_info), _vp]),
    "qcd_workspace_bytes_batched": (_sz, [_i, ctypes.POINTER(_vp), ctypes.POINTER(qcd_solver_opts)]),
    "qcd_cg_solve_batched": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                  ctypes.POINTER(_vp), ctypes.POINTER(_d), _d, _i, ctypes.POINTER(qcd_solver_opts),
                                  _vp, ctypes.POINTER(qcd_solve_info), _vp]),
    "qcd_workspace_bytes_full": (_sz, [_vp, ctypes.POINTER(qcd_solver_opts)]),
    "qcd_solve_full": (_i, [_vp, _vp, _vp, _d, _d, _i, ctypes.POINTER(qcd_solver_opts), _vp,
                            ctypes.POINTER(qcd_solve_info), _vp]),
    "qcd_fermion_force": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "qcd_device_span_bytes": (_sz, [_vp]),
    "qcd_wilson_field_bytes": (_sz, [_vp, _i]),
    "qcd_wilson_links_bytes": (_sz, [_vp, _i]),
    "qcd_wilson_load_links": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qcd_wilson_pack_field": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qcd_wilson_unpack_field": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qcd_wilson_op": (_i, [_vp, _vp, _vp, _d, _i, _i, _vp]),
    "qcd_wilson_op_mrhs": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, _vp]),
    "qcd_wilson_workspace_bytes": (_sz, [_vp, ctypes.POINTER(qcd_solver_opts), _i]),
    "qcd_wilson_cgnr": (_i, [_vp, _vp, _vp, _d, _d, _i, ctypes.POINTER(qcd_solver_opts), _vp,
                             ctypes.POINTER(qcd_solve_info), _vp]),
    "qcd_wilson_cgnr_mrhs": (_i, [_vp, _i, _vp, _vp, _d, _d, _i, ctypes.POINTER(qcd_solver_opts), _vp,
                                  ctypes.POINTER(qcd_solve_info), _vp]),
    "qcd_tune_mrhs": (_i, [_vp, _i, _vp, _vp, _d, ctypes.POINTER(qcd_solver_opts), _vp, ctypes.c_char_p,
                           ctypes.POINTER(_i), _vp]),
    "qcd_tune_batched": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_d),
                              _d, _i, ctypes.POINTER(qcd_solver_opts), _vp, ctypes.c_char_p, ctypes.POINTER(_i),
                              ctypes.POINTER(_i), _vp]),
    "qcd_tune_load": (_i, [ctypes.c_char_p]),
    "qcd_cg_solve_mrhs": (_i, [_vp, _i, _vp, _vp, _d, _d, _i, ctypes.POINTER(qcd_solver_opts), _vp, _vp,
                               ctypes.POINTER(qcd_solve_info), _vp]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc: int, where: str, ok=(QCD_OK,)) -> int:
    if rc not in ok:
        msg = _lib.qcd_last_error().decode() or _lib.qcd_status_string(rc).decode()
        raise QcdError(rc, where, msg)
    return rc


# ---------------------------------------------------------------- thin wrappers (same names)

def qcd_version() -> str:
    return _lib.qcd_version().decode()


def qcd_status_string(status: int) -> str:
    return _lib.qcd_status_string(status).decode()


def qcd_lattice_create(L0: int, L1: int, L2: int, L3: int) -> int:
    h = _vp()
    _check(_lib.qcd_lattice_create(L0, L1, L2, L3, ctypes.byref(h)), "qcd_lattice_create")
    return h.value


def qcd_lattice_destroy(lat: int) -> None:
    _check(_lib.qcd_lattice_destroy(lat), "qcd_lattice_destroy")


def qcd_lattice_set_tbc(lat: int, sign: int) -> None:
    _check(_lib.qcd_lattice_set_tbc(lat, sign), "qcd_lattice_set_tbc")


def qcd_lattice_device(lat: int) -> int:
    return _lib.qcd_lattice_device(lat)


def qcd_field_bytes(lat: int, prec: int) -> int:
    return _lib.qcd_field_bytes(lat, prec)


def qcd_links_bytes(lat: int, prec: int, recon: int) -> int:
    return _lib.qcd_links_bytes(lat, prec, recon)


def qcd_solver_opts_default() -> qcd_solver_opts:
    o = qcd_solver_opts()
    _lib.qcd_solver_opts_default(ctypes.byref(o))
    return o


def qcd_workspace_bytes(lat: int, opts: qcd_solver_opts | None = None, nrhs: int = 1) -> int:
    return _lib.qcd_workspace_bytes(lat, ctypes.byref(opts) if opts is not None else None, nrhs)


def qcd_load_links(lat, links_dev, packed_dev, prec, recon, stream=None):
    return _check(_lib.qcd_load_links(lat, _ptr(links_dev), _ptr(packed_dev), prec, recon, _stream(stream)),
                  "qcd_load_links")


def qcd_pack_field(lat, packed_dev, canonical_dev, parity, prec, stream=None):
    return _check(_lib.qcd_pack_field(lat, _ptr(packed_dev), _ptr(canonical_dev), parity, prec, _stream(stream)),
                  "qcd_pack_field")


def qcd_unpack_field(lat, canonical_dev, packed_dev, parity, prec, stream=None):
    return _check(_lib.qcd_unpack_field(lat, _ptr(canonical_dev), _ptr(packed_dev), parity, prec, _stream(stream)),
                  "qcd_unpack_field")


def qcd_dslash(lat, out_dev, in_dev, out_parity, prec, stream=None):
    return _check(_lib.qcd_dslash(lat, _ptr(out_dev), _ptr(in_dev), out_parity, prec, _stream(stream)),
                  "qcd_dslash")


def qcd_dslash_mrhs(lat, out_dev, in_dev, nrhs, out_parity, prec, stream=None):
    return _check(_lib.qcd_dslash_mrhs(lat, _ptr(out_dev), _ptr(in_dev), nrhs, out_parity, prec, _stream(stream)),
                  "qcd_dslash_mrhs")


def qcd_mdagm(lat, out_dev, in_dev, mass, prec, tmp_dev, stream=None):
    return _check(_lib.qcd_mdagm(lat, _ptr(out_dev), _ptr(in_dev), float(mass), prec, _ptr(tmp_dev),
                                 _stream(stream)), "qcd_mdagm")


def qcd_mdagm_noalloc(lat, out_dev, in_dev, mass, prec, stream=None):
    """qcd_mdagm without caller scratch: the library's built-in 16 MiB device array holds the
    intermediate field, for callers that cannot allocate device memory."""
    return _check(_lib.qcd_mdagm_noalloc(lat, _ptr(out_dev), _ptr(in_dev), float(mass), prec, _stream(stream)),
                  "qcd_mdagm_noalloc")


def qcd_cg_solve(lat, x_dev, b_dev, mass, tol, max_iter, opts, workspace_dev, y_dev=None, stream=None,
                 raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    """Returns (status, info dict). Convergence failures are returned, not raised."""
    info = qcd_solve_info()
    rc = _lib.qcd_cg_solve(lat, _ptr(x_dev), _ptr(b_dev), float(mass), float(tol), int(max_iter),
                           ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev), _ptr(y_dev),
                           ctypes.byref(info), _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_cg_solve")
    return rc, info.as_dict()


def qcd_cg_solve_mrhs(lat, nrhs, x_dev, b_dev, mass, tol, max_iter, opts, workspace_dev, y_dev=None, stream=None,
                      raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    """Returns (status, [info dict per RHS])."""
    infos = (qcd_solve_info * max(int(nrhs), 1))()
    rc = _lib.qcd_cg_solve_mrhs(lat, int(nrhs), _ptr(x_dev), _ptr(b_dev), float(mass), float(tol), int(max_iter),
                                ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev), _ptr(y_dev),
                                infos, _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_cg_solve_mrhs")
    return rc, [i.as_dict() for i in infos]


def _ptr_array(items):
    return (_vp * len(items))(*[_ptr(t) for t in items])


def qcd_workspace_bytes_batched(lats, opts=None) -> int:
    return _lib.qcd_workspace_bytes_batched(len(lats), _ptr_array(lats), ctypes.byref(opts) if opts is not None else None)


def qcd_cg_solve_batched(lats, x_devs, b_devs, y_devs, masses, tol, max_iter, opts, workspace_dev, stream=None,
                         raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    """Returns (status, [info dict per lattice])."""
    n = len(lats)
    infos = (qcd_solve_info * max(n, 1))()
    ys = _ptr_array(y_devs) if y_devs is not None else None
    m = (_d * n)(*[float(v) for v in masses])
    rc = _lib.qcd_cg_solve_batched(n, _ptr_array(lats), _ptr_array(x_devs), _ptr_array(b_devs), ys, m, float(tol),
                                   int(max_iter), ctypes.byref(opts) if opts is not None else None,
                                   _ptr(workspace_dev), infos, _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_cg_solve_batched")
    return rc, [infos[i].as_dict() for i in range(n)]


def qcd_workspace_bytes_full(lat, opts=None) -> int:
    return _lib.qcd_workspace_bytes_full(lat, ctypes.byref(opts) if opts is not None else None)


def qcd_solve_full(lat, x_dev, b_dev, mass, tol, max_iter, opts, workspace_dev, stream=None,
                   raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    """x = M^-1 b on both parities. Returns (status, info dict)."""
    info = qcd_solve_info()
    rc = _lib.qcd_solve_full(lat, _ptr(x_dev), _ptr(b_dev), float(mass), float(tol), int(max_iter),
                             ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev),
                             ctypes.byref(info), _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_solve_full")
    return rc, info.as_dict()


def qcd_fermion_force(lat, force_dev, links_dev, x_dev, y_dev, stream=None):
    """force[n][mu] = G_mu(n), the traceless Hermitian derivative of phi^dagger A^-1 phi (x even, y odd)."""
    return _check(_lib.qcd_fermion_force(lat, _ptr(force_dev), _ptr(links_dev), _ptr(x_dev), _ptr(y_dev),
                                         _stream(stream)), "qcd_fermion_force")


QCD_WILSON_DSLASH, QCD_WILSON_M, QCD_WILSON_MDAG = 0, 1, 2


def qcd_device_span_bytes(ptr) -> int:
    return _lib.qcd_device_span_bytes(_ptr(ptr))


def qcd_wilson_field_bytes(lat, prec) -> int:
    return _lib.qcd_wilson_field_bytes(lat, prec)


def qcd_wilson_links_bytes(lat, prec) -> int:
    return _lib.qcd_wilson_links_bytes(lat, prec)


def qcd_wilson_load_links(lat, links_dev, packed_dev, prec, stream=None):
    return _check(_lib.qcd_wilson_load_links(lat, _ptr(links_dev), _ptr(packed_dev), prec, _stream(stream)),
                  "qcd_wilson_load_links")


def qcd_wilson_pack_field(lat, packed_dev, canonical_dev, prec, stream=None):
    return _check(_lib.qcd_wilson_pack_field(lat, _ptr(packed_dev), _ptr(canonical_dev), prec, _stream(stream)),
                  "qcd_wilson_pack_field")


def qcd_wilson_unpack_field(lat, canonical_dev, packed_dev, prec, stream=None):
    return _check(_lib.qcd_wilson_unpack_field(lat, _ptr(canonical_dev), _ptr(packed_dev), prec, _stream(stream)),
                  "qcd_wilson_unpack_field")


def qcd_wilson_op(lat, out_dev, in_dev, kappa, op, prec, stream=None):
    return _check(_lib.qcd_wilson_op(lat, _ptr(out_dev), _ptr(in_dev), float(kappa), int(op), prec, _stream(stream)),
                  "qcd_wilson_op")


def qcd_wilson_op_mrhs(lat, out_dev, in_dev, nrhs, kappa, op, prec, stream=None):
    return _check(_lib.qcd_wilson_op_mrhs(lat, _ptr(out_dev), _ptr(in_dev), int(nrhs), float(kappa), int(op), prec,
                                          _stream(stream)), "qcd_wilson_op_mrhs")


def qcd_wilson_workspace_bytes(lat, opts=None, nrhs=1) -> int:
    return _lib.qcd_wilson_workspace_bytes(lat, ctypes.byref(opts) if opts is not None else None, int(nrhs))


def qcd_wilson_cgnr(lat, x_dev, b_dev, kappa, tol, max_iter, opts, workspace_dev, stream=None,
                    raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    info = qcd_solve_info()
    rc = _lib.qcd_wilson_cgnr(lat, _ptr(x_dev), _ptr(b_dev), float(kappa), float(tol), int(max_iter),
                              ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev),
                              ctypes.byref(info), _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_wilson_cgnr")
    return rc, info.as_dict()


def qcd_wilson_cgnr_mrhs(lat, nrhs, x_dev, b_dev, kappa, tol, max_iter, opts, workspace_dev, stream=None,
                         raise_on=(QCD_ERR_INVALID_ARG, QCD_ERR_CUDA, QCD_ERR_UNSUPPORTED, QCD_ERR_NO_LINKS)):
    """Returns (status, [info dict per RHS])."""
    infos = (qcd_solve_info * max(int(nrhs), 1))()
    rc = _lib.qcd_wilson_cgnr_mrhs(lat, int(nrhs), _ptr(x_dev), _ptr(b_dev), float(kappa), float(tol), int(max_iter),
                                   ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev), infos,
                                   _stream(stream))
    if rc in raise_on:
        _check(rc, "qcd_wilson_cgnr_mrhs")
    return rc, [i.as_dict() for i in infos]


def qcd_tune_mrhs(lat, nrhs, x_dev, b_dev, mass, opts, workspace_dev, cache_path=None, stream=None) -> int:
    best = _i()
    _check(_lib.qcd_tune_mrhs(lat, int(nrhs), _ptr(x_dev), _ptr(b_dev), float(mass),
                              ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev),
                              cache_path.encode() if cache_path else None, ctypes.byref(best), _stream(stream)),
           "qcd_tune_mrhs")
    return best.value


def qcd_tune_batched(lats, x_devs, b_devs, masses, tol, max_iter, opts, workspace_dev, cache_path=None, stream=None):
    n = len(lats)
    c, blk = _i(), _i()
    m = (_d * n)(*[float(v) for v in masses])
    _check(_lib.qcd_tune_batched(n, _ptr_array(lats), _ptr_array(x_devs), _ptr_array(b_devs), m, float(tol),
                                 int(max_iter), ctypes.byref(opts) if opts is not None else None, _ptr(workspace_dev),
                                 cache_path.encode() if cache_path else None, ctypes.byref(c), ctypes.byref(blk),
                                 _stream(stream)), "qcd_tune_batched")
    return c.value, blk.value


def qcd_tune_load(cache_path: str) -> None:
    _check(_lib.qcd_tune_load(cache_path.encode()), "qcd_tune_load")


# ---------------------------------------------------------------- convenience owner object

class Lattice:
    """A lattice handle plus torch-owned device buffers for its packed links and workspaces."""

    def __init__(self, dims, tbc: int = -1):
        import torch  # device memory and streams only
        self._torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.Vh = self.V // 2
        self.handle = qcd_lattice_create(*self.dims)
        if tbc != -1:
            qcd_lattice_set_tbc(self.handle, tbc)
        self._links = {}
        self._ws = {}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.qcd_lattice_destroy(h)
            self.handle = None

    def empty_bytes(self, nbytes: int):
        # 256-byte aligned device buffer (the caching allocator aligns to 512 B)
        return self._torch.empty(max(int(nbytes), 1), dtype=self._torch.uint8, device="cuda")

    def field(self, prec: int, nrhs: int = 1):
        return self.empty_bytes(qcd_field_bytes(self.handle, prec) * nrhs)

    def load_links(self, links_canon_dev, prec: int = QCD_PREC_DOUBLE, recon: int = 18, stream=None):
        buf = self.empty_bytes(qcd_links_bytes(self.handle, prec, recon))
        qcd_load_links(self.handle, links_canon_dev, buf, prec, recon, stream)
        self._links[prec] = buf
        return buf

    def workspace(self, opts: qcd_solver_opts, nrhs: int = 1):
        n = qcd_workspace_bytes(self.handle, opts, nrhs)
        key = (opts.prec_inner, nrhs)
        if key not in self._ws or self._ws[key].numel() < n:
            self._ws[key] = self.empty_bytes(n)
        return self._ws[key]
