"""Row-partitioned product: binding of the ``sp_dist_*`` calls of the C ABI.

GHOST distributes the system matrix row-wise over processes (Sec. "Data
parallelism"), with a work share per process (Sec. "Heterogeneous
execution"); each process keeps its rows, its remote columns compressed into
a halo numbered after its own rows, and the product overlaps the halo
exchange with the local part (the task-mode SpMV of Sec. "Resource
management").  The plan, the column split and both device steps (halo pack,
two-pass product) are the library's; this module marshals arguments and
hands the exchange and the sum of the dot products to a communicator:

* :class:`TorchComm` -- ``torch.distributed`` (NCCL between GPUs, gloo on
  the CPU): ``all_to_all_single`` for the halo rows and the send lists,
  ``all_reduce`` for the 3 w dot sums.
* :class:`LocalWorld` -- every part in one process on one device (the parts
  run one after the other; the exchange is device-to-device copies).  No
  kernel ever waits for another part's kernel.

There is no CPU path: the product calls need the CUDA library.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import sellcs
from .sellcs import _ptr, _stream, check, lib


def partition(nrows: int, rowptr=None, nparts: int = 1, share=None, by_nnz: bool = True) -> np.ndarray:
    """Row bounds (int64[nparts + 1]) of contiguous blocks whose work (nonzeros
    when ``by_nnz``, else rows) follows ``share`` (sp_dist_partition)."""
    b = np.empty(nparts + 1, np.int64)
    rp = None if rowptr is None else np.ascontiguousarray(rowptr, np.int64)
    sh = None if share is None else np.ascontiguousarray(share, np.float64)
    check(lib().sp_dist_partition(int(nrows), _ptr(rp), int(nparts), _ptr(sh), 1 if by_nnz else 0, _ptr(b)),
          "sp_dist_partition")
    return b


def rows_of(A, r0: int, r1: int):
    """Rows [r0, r1) of a CSR object: (rowptr from 0, global int64 columns, values)."""
    a, b = int(A.rowptr[r0]), int(A.rowptr[r1])
    rp = np.ascontiguousarray(A.rowptr[r0:r1 + 1] - a, np.int64)
    return rp, np.ascontiguousarray(A.col[a:b], np.int64), np.ascontiguousarray(A.val[a:b], np.float64)


class DistPlan:
    """One process's plan (sp_dist_plan): its rows, the halo, the send list."""

    def __init__(self, nglobal: int, bounds, rank: int, rowptr, gcol):
        self._lib = lib()
        self.bounds = np.ascontiguousarray(bounds, np.int64)
        self.nranks = len(self.bounds) - 1
        self.rank = int(rank)
        self.rowptr = np.ascontiguousarray(rowptr, np.int64)
        gcol = np.ascontiguousarray(gcol, np.int64)
        h = ct.c_void_p()
        check(self._lib.sp_dist_plan_create(ct.byref(h), int(nglobal), self.nranks, _ptr(self.bounds), self.rank,
                                            _ptr(self.rowptr), _ptr(gcol)), "sp_dist_plan_create")
        self.handle = h

    def info(self) -> dict:
        v = [ct.c_int64() for _ in range(5)]
        check(self._lib.sp_dist_plan_info(self.handle, *[ct.byref(q) for q in v]), "sp_dist_plan_info")
        return dict(zip(("nloc", "nhalo", "nnz_local", "nnz_remote", "nsend"), (q.value for q in v)))

    def halo(self):
        """(global row of each halo entry, halo entries owned by each rank)."""
        i = self.info()
        g = np.empty(i["nhalo"], np.int64)
        rc = np.empty(self.nranks, np.int64)
        check(self._lib.sp_dist_plan_halo(self.handle, _ptr(g), _ptr(rc)), "sp_dist_plan_halo")
        return g, rc

    def columns(self) -> np.ndarray:
        """Local column of every entry (CSR order), in [0, nloc + nhalo)."""
        c = np.empty(int(self.rowptr[-1]), np.int32)
        check(self._lib.sp_dist_plan_columns(self.handle, _ptr(c)), "sp_dist_plan_columns")
        return c

    def split(self, val):
        """((rowptr, col, val) of the local part, (rowptr, col, val) of the remote part)."""
        i = self.info()
        val = np.ascontiguousarray(val, np.float64)
        n = i["nloc"]
        loc = (np.empty(n + 1, np.int64), np.empty(i["nnz_local"], np.int32), np.empty(i["nnz_local"]))
        rem = (np.empty(n + 1, np.int64), np.empty(i["nnz_remote"], np.int32), np.empty(i["nnz_remote"]))
        check(self._lib.sp_dist_plan_split(self.handle, _ptr(val), *[_ptr(a) for a in loc], *[_ptr(a) for a in rem]),
              "sp_dist_plan_split")
        return loc, rem

    def set_sends(self, send_counts, send_gidx):
        sc = np.ascontiguousarray(send_counts, np.int64)
        sg = np.ascontiguousarray(send_gidx, np.int64)
        check(self._lib.sp_dist_plan_set_sends(self.handle, _ptr(sc), _ptr(sg)), "sp_dist_plan_set_sends")

    def sends(self):
        """(rows sent to each rank, local row of each sent row)."""
        i = self.info()
        sc = np.empty(self.nranks, np.int64)
        sl = np.empty(max(i["nsend"], 0), np.int32)
        check(self._lib.sp_dist_plan_sends(self.handle, _ptr(sc), _ptr(sl)), "sp_dist_plan_sends")
        return sc, sl

    def exchange_sends(self, comm):
        """Tell every owner which of its rows this process needs (one
        all-to-all of the counts, one of the global indices), and store what
        the others need from it."""
        import torch
        g, rc = self.halo()
        recv_counts = comm.alltoall_counts(rc)
        send_gidx = torch.empty(int(recv_counts.sum()), dtype=torch.int64, device=comm.index_device)
        comm.alltoallv(torch.from_numpy(g).to(comm.index_device), [int(c) for c in rc], send_gidx,
                       [int(c) for c in recv_counts])
        self.set_sends(recv_counts, send_gidx.cpu().numpy())

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sp_dist_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split_opts(opts: sellcs.sp_spmv_opts):
    """The two passes of the overlapped product (sp_dist_split_opts)."""
    p1, p2 = sellcs.sp_spmv_opts(), sellcs.sp_spmv_opts()
    check(lib().sp_dist_split_opts(ct.byref(opts), ct.byref(p1), ct.byref(p2)), "sp_dist_split_opts")
    return p1, p2


class TorchComm:
    """Exchange and sums over a ``torch.distributed`` process group."""

    def __init__(self, group=None, device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        nccl = dist.get_backend(group) == "nccl"
        self.index_device = device if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu"))

    def alltoall_counts(self, counts) -> np.ndarray:
        import torch
        s = torch.as_tensor(np.asarray(counts, np.int64)).to(self.index_device)
        r = torch.empty_like(s)
        self.dist.all_to_all_single(r, s, group=self.group)
        return r.cpu().numpy()

    def alltoallv(self, send, send_counts, recv, recv_counts):
        """Rows of ``send`` (split by send_counts, rank after rank) into
        ``recv`` (split by recv_counts)."""
        self.dist.all_to_all_single(recv, send, list(recv_counts), list(send_counts), group=self.group)

    def allreduce_sum(self, t):
        self.dist.all_reduce(t, group=self.group)


class DistMatrix:
    """One process's rows on the device.

    ``mode="overlap"``: the local part and the remote part as two SELL-C-sigma
    matrices; the halo exchange runs on a side stream while the local pass
    runs (sp_dist_spmv).  ``mode="no_overlap"``: one matrix over the extended
    columns, the exchange first, then one product (the paper's "No Overlap"
    variant)."""

    def __init__(self, plan: DistPlan, val, C=32, sigma=1, dtype="f64", mode="overlap", stream=None):
        import torch
        assert mode in ("overlap", "no_overlap")
        self.plan = plan
        self.mode = mode
        i = plan.info()
        if i["nsend"] < 0:
            raise ValueError("the plan's send list is not set (exchange_sends)")
        self.nloc, self.nhalo = i["nloc"], i["nhalo"]
        self.send_counts, _ = plan.sends()
        _, self.recv_counts = plan.halo()
        ncols = self.nloc + self.nhalo
        if mode == "overlap":
            (rl, cl, vl), (rr, cr, vr) = plan.split(val)
            self.A_loc = sellcs.SellMatrix(_Csr(self.nloc, self.nloc, rl, cl, vl), C=C, sigma=sigma, dtype=dtype,
                                           stream=stream)
            self.A_rem = sellcs.SellMatrix(_Csr(self.nloc, ncols, rr, cr, vr), C=C, sigma=sigma, dtype=dtype,
                                           stream=stream)
        else:
            self.A_ext = sellcs.SellMatrix(_Csr(self.nloc, ncols, plan.rowptr, plan.columns(),
                                                np.ascontiguousarray(val, np.float64)), C=C, sigma=sigma,
                                           dtype=dtype, stream=stream)
        self.comm_stream = torch.cuda.Stream()
        self._send = {}

    def send_buffer(self, w, dtype, device):
        import torch
        key = (w, dtype)
        if key not in self._send:
            self._send[key] = torch.empty((int(self.send_counts.sum()), w), dtype=dtype, device=device)
        return self._send[key]

    def new_x(self, w=1, dtype=None, device=None):
        """A zeroed (nloc + nhalo) x w block vector: rows 0..nloc-1 for the
        caller's x, the rest for the halo."""
        import torch
        return torch.zeros((self.nloc + self.nhalo, w), dtype=dtype or torch.float64, device=device or "cuda")

    def pack(self, x_ext, stream=None):
        """Gather the rows the other processes need into the send buffer."""
        buf = self.send_buffer(x_ext.shape[1], x_ext.dtype, x_ext.device)
        hx = sellcs.sp_dense_view(x_ext)
        try:
            check(lib().sp_dist_pack(self.plan.handle, hx, _ptr(buf), _stream(stream)), "sp_dist_pack")
        finally:
            lib().sp_dense_destroy(hx, None)
        return buf

    def product(self, x_ext, y, *, halo_ready=None, alpha=None, gamma=None, beta=None, dot_yy=False, dot_xy=False,
                dot_xx=False, z=None, delta=None, eta=None, dot=None, stream=None):
        """This process's product with its halo in x_ext (rows nloc..) ready,
        or arriving by the CUDA event ``halo_ready`` (overlap mode); the dots
        in ``dot`` are this process's partial sums."""
        import torch
        w = x_ext.shape[1]
        if (dot_yy or dot_xy or dot_xx) and dot is None:
            dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device=x_ext.device)
        hx, hy = sellcs.sp_dense_view(x_ext), sellcs.sp_dense_view(y)
        hz = sellcs.sp_dense_view(z) if z is not None else None
        try:
            o, keep = sellcs.make_opts(w, alpha=alpha, gamma=gamma, beta=beta, dot_yy=dot_yy, dot_xy=dot_xy,
                                       dot_xx=dot_xx, z_handle=hz, delta=delta, eta=eta,
                                       dot_ptr=_ptr(dot) if dot is not None else None)
            if self.mode == "overlap":
                ev = ct.c_void_p(halo_ready.cuda_event) if halo_ready is not None else None
                check(lib().sp_dist_spmv(hy, self.A_loc.handle, self.A_rem.handle, hx, ct.byref(o), ev,
                                         _stream(stream)), "sp_dist_spmv")
            else:
                if halo_ready is not None:
                    (stream or torch.cuda.current_stream()).wait_event(halo_ready)
                check(lib().sp_spmv(hy, self.A_ext.handle, hx, ct.byref(o), _stream(stream)), "sp_spmv")
        finally:
            for h in (hx, hy, hz):
                if h is not None:
                    lib().sp_dense_destroy(h, None)
        return dot

    def spmv(self, comm, x_ext, y, **kw):
        """The distributed product through ``comm`` (a :class:`TorchComm`):
        pack and exchange the halo on a side stream, the product on the
        current stream (overlapping the local pass in overlap mode), then the
        sum of the dots over processes.  Returns the summed dots (or None)."""
        import torch
        cur = torch.cuda.current_stream()
        self.comm_stream.wait_stream(cur)
        with torch.cuda.stream(self.comm_stream):
            buf = self.pack(x_ext, self.comm_stream)
            comm.alltoallv(buf, self.send_counts, x_ext[self.nloc:], self.recv_counts)
            ready = torch.cuda.Event()
            ready.record(self.comm_stream)
        dot = self.product(x_ext, y, halo_ready=ready, stream=cur, **kw)
        x_ext.record_stream(self.comm_stream)
        if dot is not None:
            comm.allreduce_sum(dot)
        return dot

    def close(self):
        for n in ("A_loc", "A_rem", "A_ext"):
            m = getattr(self, n, None)
            if m is not None:
                m.close()


class _Csr:
    def __init__(self, nrows, ncols, rowptr, col, val):
        self.nrows, self.ncols, self.rowptr, self.col, self.val = int(nrows), int(ncols), rowptr, col, val


class LocalWorld:
    """Every part of a row partition in this process, on the current device.

    The parts run one after the other on one stream; the halo exchange is a
    copy of each sender's packed rows into the receiver's halo rows.  Used to
    check and time the partitioned product on one GPU."""

    def __init__(self, A, nparts, C=32, sigma=1, dtype="f64", mode="overlap", share=None, by_nnz=True):
        self.bounds = partition(A.nrows, A.rowptr, nparts, share, by_nnz)
        self.plans, self.mats = [], []
        for r in range(nparts):
            rp, gc, _ = rows_of(A, self.bounds[r], self.bounds[r + 1])
            self.plans.append(DistPlan(A.nrows, self.bounds, r, rp, gc))
        halos = [p.halo() for p in self.plans]
        for q, p in enumerate(self.plans):  # q's sends: the halo entries of every other part in q's rows
            counts, lists = [], []
            for r in range(nparts):
                g = halos[r][0]
                sel = g[(g >= self.bounds[q]) & (g < self.bounds[q + 1])] if r != q else g[:0]
                counts.append(sel.size)
                lists.append(sel)
            p.set_sends(np.array(counts, np.int64), np.concatenate(lists) if lists else np.zeros(0, np.int64))
        for r in range(nparts):
            _, _, v = rows_of(A, self.bounds[r], self.bounds[r + 1])
            self.mats.append(DistMatrix(self.plans[r], v, C=C, sigma=sigma, dtype=dtype, mode=mode))

    def scatter(self, X):
        """Per part, an extended x (own rows from the global X, zero halo)."""
        import torch
        X = torch.as_tensor(X)
        X2 = X.reshape(X.shape[0], -1)
        out = []
        for r, m in enumerate(self.mats):
            xe = m.new_x(X2.shape[1], X2.dtype, "cuda")
            xe[:m.nloc].copy_(X2[self.bounds[r]:self.bounds[r + 1]])
            out.append(xe)
        return out

    def exchange(self, xs):
        """Pack every part's sends and copy them into the receivers' halos."""
        bufs = [m.pack(x) for m, x in zip(self.mats, xs)]
        n = len(self.mats)
        send_off = [np.concatenate([[0], np.cumsum(m.send_counts)]) for m in self.mats]
        recv_off = [np.concatenate([[0], np.cumsum(m.recv_counts)]) for m in self.mats]
        for q in range(n):          # receiver
            for r in range(n):      # sender
                c = int(self.mats[q].recv_counts[r])
                if c == 0:
                    continue
                assert int(self.mats[r].send_counts[q]) == c
                s0 = int(send_off[r][q])
                d0 = self.mats[q].nloc + int(recv_off[q][r])
                xs[q][d0:d0 + c].copy_(bufs[r][s0:s0 + c])

    def spmv(self, xs, ys, zs=None, **kw):
        """Exchange, every part's product, and the sum of the dots over the
        parts (in part order).  Returns the summed dots (or None)."""
        self.exchange(xs)
        total = None
        for r, m in enumerate(self.mats):
            d = m.product(xs[r], ys[r], z=None if zs is None else zs[r], **kw)
            if d is not None:
                total = d.clone() if total is None else total + d
        return total
