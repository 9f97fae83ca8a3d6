"""Helpers for the GPU parity tests: move seeded host inputs to the device and run the C-ABI."""
import numpy as np

from paper_1311_2719_gb300 import qcd as Q

PRECS = {"double": (Q.QCD_PREC_DOUBLE, 18), "single18": (Q.QCD_PREC_SINGLE, 18),
         "single12": (Q.QCD_PREC_SINGLE, 12), "half12": (Q.QCD_PREC_HALF, 12), "df64": (Q.QCD_PREC_DF64, 18)}
# relative-L2 bars of the half-lattice operator against the FP64 oracle (df64 is held to FP64's)
TOL = {"double": 1e-12, "single18": 1e-5, "single12": 1e-5, "half12": 5e-3, "df64": 1e-12}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.cpu().numpy()


class Rig:
    """A lattice with its links loaded at the requested (precision, recon) pairs."""

    def __init__(self, dims, U, precs=("double",), tbc=-1):
        import torch
        self.torch = torch
        self.dims = tuple(dims)
        self.lat = Q.Lattice(dims, tbc=tbc)
        self.h = self.lat.handle
        self.V = self.lat.V
        self.U_dev = dev(U)
        for name in precs:
            p, r = PRECS[name]
            self.lat.load_links(self.U_dev, p, r)

    def zeros_canon(self, nrhs=None):
        shape = (self.V, 3) if nrhs is None else (nrhs, self.V, 3)
        return self.torch.zeros(shape, dtype=self.torch.complex128, device="cuda")

    def pack(self, x_canon_dev, parity, prec):
        f = self.lat.field(prec)
        Q.qcd_pack_field(self.h, f, x_canon_dev, parity, prec)
        return f

    def unpack(self, f, parity, prec, out=None):
        o = self.zeros_canon() if out is None else out
        Q.qcd_unpack_field(self.h, o, f, parity, prec)
        return o

    def dslash(self, x, out_parity, name="double"):
        prec = PRECS[name][0]
        fin = self.pack(dev(x), 1 - out_parity, prec)
        fout = self.lat.field(prec)
        Q.qcd_dslash(self.h, fout, fin, out_parity, prec)
        return host(self.unpack(fout, out_parity, prec))

    def mdagm(self, x, mass, name="double"):
        prec = PRECS[name][0]
        fin = self.pack(dev(x), Q.QCD_EVEN, prec)
        fout = self.lat.field(prec)
        tmp = self.lat.field(prec)
        Q.qcd_mdagm(self.h, fout, fin, mass, prec, tmp)
        return host(self.unpack(fout, Q.QCD_EVEN, prec))

    def dslash_mrhs(self, xs, out_parity, name="double"):
        prec = PRECS[name][0]
        n = len(xs)
        fb = Q.qcd_field_bytes(self.h, prec)
        fin = self.lat.field(prec, n)
        fout = self.lat.field(prec, n)
        for r in range(n):
            Q.qcd_pack_field(self.h, fin.data_ptr() + r * fb, dev(xs[r]), 1 - out_parity, prec)
        Q.qcd_dslash_mrhs(self.h, fout, fin, n, out_parity, prec)
        outs = []
        for r in range(n):
            o = self.zeros_canon()
            Q.qcd_unpack_field(self.h, o, fout.data_ptr() + r * fb, out_parity, prec)
            outs.append(host(o))
        return np.stack(outs)

    def cg(self, b, mass, tol=1e-10, max_iter=10000, inner="double", use_graph=1, check_interval=8,
           stream=None, want_y=True, staged=0):
        opts = Q.qcd_solver_opts_default()
        opts.prec_inner, opts.recon_inner = PRECS[inner]
        opts.use_graph = use_graph
        opts.staged = staged
        opts.check_interval = check_interval
        ws = self.lat.workspace(opts)
        bd = dev(b)
        x = self.zeros_canon()
        y = self.zeros_canon() if want_y else None
        s = stream if stream is not None else self.torch.cuda.Stream()
        s.wait_stream(self.torch.cuda.current_stream())
        with self.torch.cuda.stream(s):
            rc, info = Q.qcd_cg_solve(self.h, x, bd, mass, tol, max_iter, opts, ws, y, stream=s)
        s.synchronize()
        return rc, info, host(x), (host(y) if want_y else None)
