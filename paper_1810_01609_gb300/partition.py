"""T-partitioned lattices (Sec. "Current State of the Art": the radius-one stencil is
decomposed across GPUs; the faces of each partition are exchanged while its interior is
computed).  All arithmetic runs in libmdwf; this module splits fields, drives the
partitions and moves faces.

* `split_links` / `split_t` / `join_t`: a global gauge field or 5D field as per-partition
  arrays (the links with the lower neighbour's last timeslice in front, as
  mdwf_load_gauge of a partitioned context takes them).
* `PartitionedLattice`: the partitions of one lattice as contexts of this process, grouped
  for the library's in-process face exchange and driven one host thread and one stream
  each.
* `TorchFaceExchange`: the face exchange between processes, one partition per rank, with
  torch.distributed point-to-point messages (NCCL on device buffers, or gloo through host
  copies); `exchange()` is the host-side routing alone.
"""
import threading

import numpy as np

from . import _lib as L
from .api import Context


def split_links(U, t_ranks):
    """Global links [T][Z][Y][X][4][3][3] -> t_ranks arrays of T/t_ranks + 1 timeslices:
    the lower neighbour's last timeslice (periodically), then the partition's own."""
    T = U.shape[0]
    if T % t_ranks:
        raise ValueError("T must be a multiple of t_ranks")
    tl = T // t_ranks
    return [np.ascontiguousarray(U[[(r * tl - 1) % T] + list(range(r * tl, (r + 1) * tl))]) for r in range(t_ranks)]


def split_t(field, t_ranks, t_axis):
    """A field's slabs along its T axis (views for torch tensors / numpy arrays)."""
    T = field.shape[t_axis]
    tl = T // t_ranks
    idx = [slice(None)] * field.ndim
    out = []
    for r in range(t_ranks):
        idx[t_axis] = slice(r * tl, (r + 1) * tl)
        out.append(field[tuple(idx)])
    return out


def join_t(parts, t_axis):
    """Inverse of split_t (torch tensors or numpy arrays)."""
    if isinstance(parts[0], np.ndarray):
        return np.concatenate(parts, axis=t_axis)
    import torch
    return torch.cat(parts, dim=t_axis)


class PartitionedLattice:
    """The t_ranks partitions of one lattice (global dims X, Y, Z, T) as contexts of this
    process, grouped so that their faces are exchanged in-process."""

    def __init__(self, dims, Ls, t_ranks, **params):
        X, Y, Z, T = dims
        if T % t_ranks or (T // t_ranks) % 2:
            raise ValueError("each partition needs an even number of timeslices")
        self.dims, self.Ls, self.t_ranks = tuple(dims), int(Ls), int(t_ranks)
        self.local_dims = (X, Y, Z, T // t_ranks)
        self.ctx = [Context(self.local_dims, Ls, t_ranks=t_ranks, t_rank=r, **params) for r in range(t_ranks)]
        L.mdwf_group_partitions([c.h for c in self.ctx])

    def load_gauge(self, U):
        for c, u in zip(self.ctx, split_links(U, self.t_ranks)):
            c.load_gauge(u)

    def _parallel(self, fn):
        """fn(rank, ctx, stream) on one host thread and one CUDA stream per partition."""
        import torch
        errs = [None] * self.t_ranks
        streams = [torch.cuda.Stream() for _ in range(self.t_ranks)]

        def run(r):
            try:
                with torch.cuda.stream(streams[r]):
                    fn(r, self.ctx[r], streams[r])
                streams[r].synchronize()
            except BaseException as e:   # reported on the calling thread
                errs[r] = e

        threads = [threading.Thread(target=run, args=(r,)) for r in range(self.t_ranks)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for e in errs:
            if e is not None:
                raise e

    def apply(self, op, prec, psi, nrhs=1):
        """op on a global 5D field psi (torch, device, [nrhs][Ls][T][Z][Y][X][4][3]):
        each partition packs its slab, applies op (exchanging faces) and unpacks."""
        import torch
        prec_i = L.PRECS.get(prec, prec)
        op_i = L.OP.get(op, op) if isinstance(op, str) else op
        slabs = split_t(psi, self.t_ranks, 2)
        outs = [None] * self.t_ranks

        def work(r, ctx, stream):
            nb = ctx.field_bytes(prec_i, nrhs)
            fin = torch.zeros(nb, dtype=torch.uint8, device=psi.device)
            fout = torch.zeros(nb, dtype=torch.uint8, device=psi.device)
            src = slabs[r].contiguous()
            L.mdwf_pack(ctx.h, src, fin, prec_i, nrhs, stream)
            L.mdwf_apply(ctx.h, op_i, prec_i, fin, fout, nrhs, stream)
            out = torch.zeros_like(src)
            L.mdwf_unpack(ctx.h, fout, out, prec_i, nrhs, stream)
            outs[r] = out

        self._parallel(work)
        return join_t(outs, 2)


class TorchFaceExchange:
    """Face exchange of one partition per torch.distributed rank (rank r holds partition
    r of the group): send_lo goes to rank r-1, which receives it as its recv_hi; send_hi
    to rank r+1, received as recv_lo (periodic).  With a context, the four buffers are
    registered with it and the exchange is its callback."""

    def __init__(self, nbytes, device="cpu", ctx=None, group=None):
        import torch
        import torch.distributed as dist
        self.dist, self.group, self.nbytes = dist, group, int(nbytes)
        mk = lambda: torch.zeros(self.nbytes, dtype=torch.uint8, device=device)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self._fn = None
        if ctx is not None:
            L.mdwf_set_face_buffers(ctx, self.send_lo, self.send_hi, self.recv_lo, self.recv_hi, self.nbytes)
            self._fn = L.FACE_EXCHANGE_FN(self._callback)
            L.mdwf_set_face_exchange(ctx, self._fn)

    def exchange(self):
        """Move the faces between neighbouring ranks (blocking)."""
        dist, g = self.dist, self.group
        n = dist.get_world_size(g)
        rank = dist.get_rank(g)
        if n == 1:
            self.recv_hi.copy_(self.send_lo)
            self.recv_lo.copy_(self.send_hi)
            return
        up, down = (rank + 1) % n, (rank - 1) % n
        staged = self.send_lo.is_cuda and dist.get_backend(g) != "nccl"
        bufs = [b.cpu() if staged else b for b in (self.send_lo, self.send_hi, self.recv_lo, self.recv_hi)]
        s_lo, s_hi, r_lo, r_hi = bufs
        # tag 0: first-timeslice faces travelling down, tag 1: last-timeslice faces up
        reqs = [dist.isend(s_lo, down, group=g, tag=0), dist.irecv(r_hi, up, group=g, tag=0),
                dist.isend(s_hi, up, group=g, tag=1), dist.irecv(r_lo, down, group=g, tag=1)]
        for q in reqs:
            q.wait()
        if staged:
            self.recv_lo.copy_(r_lo)
            self.recv_hi.copy_(r_hi)

    def _callback(self, user, send_lo, send_hi, recv_lo, recv_hi, nbytes, stream):
        try:
            import torch
            if self.send_lo.is_cuda:
                torch.cuda.ExternalStream(stream).synchronize()   # faces packed
            self.exchange()
            if self.send_lo.is_cuda:
                torch.cuda.synchronize()
            return 0
        except Exception:
            return L.MDWF_ERR_CUDA
