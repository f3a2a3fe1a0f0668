"""Convenience wrapper over the C ABI: a Context owning an mdwf_ctx, with numpy / torch
inputs.  All arithmetic runs in libmdwf's CUDA kernels."""
import numpy as np

from . import _lib as L


class Context:
    def __init__(self, dims, Ls, b5=1.5, c5=0.5, M5=1.3, mf=0.05, t_bc=-1.0, recon=18, check_su3=True,
                 t_ranks=1, t_rank=0, f64_emulation=True):
        p = L.mdwf_default_params()
        for i in range(4):
            p.dims[i] = int(dims[i])
        p.Ls, p.b5, p.c5, p.M5, p.mf, p.t_bc = int(Ls), b5, c5, M5, mf, t_bc
        p.gauge_recon, p.check_su3 = int(recon), int(bool(check_su3))
        p.t_ranks, p.t_rank = int(t_ranks), int(t_rank)
        p.f64_emulation = int(bool(f64_emulation))
        self.params = p
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.h = L.mdwf_create(p)

    def __del__(self):
        if getattr(self, "h", None) is not None:
            L.mdwf_destroy(self.h)
            self.h = None

    def close(self):
        self.__del__()

    # shapes of user fields
    def shape5d(self, nrhs=None):
        X, Y, Z, T = self.dims
        s = (self.Ls, T, Z, Y, X, 4, 3)
        return s if nrhs is None else (nrhs,) + s

    def shape4d(self, nrhs=None):
        X, Y, Z, T = self.dims
        s = (T, Z, Y, X, 4, 3)
        return s if nrhs is None else (nrhs,) + s

    def load_gauge(self, links, stream=None):
        if isinstance(links, np.ndarray):
            links = np.ascontiguousarray(links, dtype=np.complex128)
        return L.mdwf_load_gauge(self.h, links, stream)

    def field_bytes(self, prec, nrhs=1):
        return L.mdwf_field_bytes(self.h, L.PRECS.get(prec, prec), nrhs)

    def solve_params(self, tol=1e-10, sloppy="f16", maxiter=100000, delta=0.05, ru_interval=100, check_interval=10,
                     use_graph=True, location=None, full_residual=False, pc_form="left"):
        sp = L.mdwf_default_solve_params()
        sp.tol, sp.maxiter, sp.sloppy_prec = tol, maxiter, L.PRECS.get(sloppy, sloppy)
        sp.delta, sp.ru_interval, sp.check_interval = delta, ru_interval, check_interval
        sp.use_graph, sp.full_residual = int(use_graph), int(full_residual)
        sp.pc_form = L.PC_FORMS.get(pc_form, pc_form)
        if location is not None:
            sp.location = location
        return sp

    def solve(self, b, sol=None, stream=None, **kw):
        """Solve D x = b for one 5D source (numpy -> host path, torch cuda -> device path)."""
        host = isinstance(b, np.ndarray)
        if host:
            b = np.ascontiguousarray(b, dtype=np.complex128)
            sol = np.empty_like(b) if sol is None else sol
        else:
            import torch
            sol = torch.empty_like(b) if sol is None else sol
        sp = self.solve_params(location=L.MDWF_HOST if host else L.MDWF_DEVICE, **kw)
        info = L.mdwf_solve(self.h, b, sol, sp, stream)
        return sol, info

    def solve_multi(self, b, sol=None, stream=None, **kw):
        host = isinstance(b, np.ndarray)
        nrhs = b.shape[0]
        if host:
            b = np.ascontiguousarray(b, dtype=np.complex128)
            sol = np.empty_like(b) if sol is None else sol
        else:
            import torch
            sol = torch.empty_like(b) if sol is None else sol
        sp = self.solve_params(location=L.MDWF_HOST if host else L.MDWF_DEVICE, **kw)
        infos = L.mdwf_solve_multi(self.h, nrhs, b, sol, sp, stream)
        return sol, infos

    def propagator(self, b4, nrhs=1, q=None, stream=None, **kw):
        """4D sources [nrhs][t][z][y][x][4][3] -> 4D propagator columns (numpy: host path,
        torch cuda: device path); returns (q, infos)."""
        if isinstance(b4, np.ndarray):
            b4 = np.ascontiguousarray(b4, dtype=np.complex128)
            q = np.empty_like(b4) if q is None else q
        else:
            import torch
            q = torch.empty_like(b4) if q is None else q
        sp = self.solve_params(**kw)
        infos = L.mdwf_propagator(self.h, nrhs, b4, q, sp, stream)
        return q, infos

    def make_source_4d(self, b4, nrhs=1, stream=None):
        out = np.empty((nrhs,) + self.shape5d(), dtype=np.complex128) if isinstance(b4, np.ndarray) else None
        if out is None:
            import torch
            out = torch.empty((nrhs,) + self.shape5d(), dtype=torch.complex128, device=b4.device)
        L.mdwf_make_source_4d(self.h, b4, out, nrhs, stream)
        return out

    def project_4d(self, y, nrhs=1, stream=None):
        if isinstance(y, np.ndarray):
            out = np.empty((nrhs,) + self.shape4d(), dtype=np.complex128)
        else:
            import torch
            out = torch.empty((nrhs,) + self.shape4d(), dtype=torch.complex128, device=y.device)
        L.mdwf_project_4d(self.h, y, out, nrhs, stream)
        return out

    def fh_source(self, q, nrhs=1, stream=None):
        out = np.empty_like(q) if isinstance(q, np.ndarray) else q.new_empty(q.shape)
        L.mdwf_fh_source(self.h, q, out, nrhs, stream)
        return out

    def contract_nucleon(self, u1, d, u2, stream=None):
        T = self.dims[3]
        if isinstance(u1, np.ndarray):
            out = np.empty(T, dtype=np.complex128)
        else:
            import torch
            out = torch.empty(T, dtype=torch.complex128, device=u1.device)
        L.mdwf_contract_nucleon(self.h, u1, d, u2, out, stream)
        return out

    def tune_entries(self):
        return L.mdwf_tune_entries(self.h)

    def launch_count(self):
        return L.mdwf_launch_count(self.h)

    def algorithmic_bytes(self):
        return L.mdwf_algorithmic_bytes(self.h)
