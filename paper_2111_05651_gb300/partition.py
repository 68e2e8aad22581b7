"""One mesh assembled by several ranks: element partition and interface-row sum.

The paper's multi-engine design (Section III-C) gives disjoint sets of
elements to concurrent engines.  Here each rank (one GPU) assembles a
disjoint set of the mesh's elements with the library, which leaves the rows
of nodes on the partition interfaces with partial sums; one sparse exchange
adds them up at the node's owner:

  setup (host, once per mesh):
    * ``rcb_partition``: recursive coordinate bisection of the element
      centroids into ``world`` parts of equal size (+-1 element);
    * ``RankPlan``: the rank's elements and the nodes they touch (its local
      mesh), the nodes it owns (a node is owned by the lowest rank whose
      elements touch it), the global CSR pattern of its owned rows, and for
      every entry and node value of its local assembly the place it goes: a
      position in its own rows, or a position in another rank's rows (then it
      is sent);
  every call (``PartitionedAssembler.assemble``; ``assemble_stabilized`` for
  the stabilised velocity block, whose entries carry twelve values -- the
  nine components of the 3x3 block, then G -- instead of four):
    1. the local assembly (``nsi_assemble`` on the rank's sub-mesh);
    2. the values of the entries of rows owned by other ranks packed into one
       send buffer (``nsi_gather_values``, a library kernel);
    3. one all-to-all of those buffers (``torch.distributed``: NCCL between
       GPUs, gloo on CPU) -- the only exchange of the path;
    4. the owned rows formed in the global pattern: the rank's own entries,
       then the entries received from each other rank in rank order, added
       by ``nsi_add_values`` (a library kernel; positions are distinct within
       one call, so plain read-add-write, and the order of the sums is fixed:
       the result does not depend on timing).

Each rank ends with A (or the stabilised Auu), G and rhs of the rows it
owns, in the global numbering and pattern (``RankPlan.own_rows``,
``own_row_ptr``, ``own_cols``).  The exchange sizes are fixed at setup.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rcb_partition(coord, lnods, parts: int) -> np.ndarray:
    """Part id (int32 [E]) of every element: recursive coordinate bisection
    of the element centroids (split along the widest extent at the weighted
    median, part counts proportional to the parts on each side)."""
    coord = np.asarray(coord, dtype=np.float64)
    lnods = np.asarray(lnods, dtype=np.int64)
    E = lnods.shape[0]
    cen = coord[lnods].mean(axis=1) if E else np.zeros((0, 3))
    out = np.zeros(E, dtype=np.int32)

    def split(idx, p0, np_):
        if np_ <= 1 or idx.size == 0:
            out[idx] = p0
            return
        ext = cen[idx].max(axis=0) - cen[idx].min(axis=0)
        ax = int(np.argmax(ext))
        left_parts = np_ // 2
        k = (idx.size * left_parts) // np_
        order = idx[np.argsort(cen[idx, ax], kind="stable")]
        split(order[:k], p0, left_parts)
        split(order[k:], p0 + left_parts, np_ - left_parts)

    split(np.arange(E), 0, parts)
    return out


def _pattern(n, lnods):
    """Sorted unique (row, col) pairs of all node pairs of the elements (CSR)."""
    ln = np.asarray(lnods, dtype=np.int64)
    if ln.size == 0:
        return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int64)
    rows = np.repeat(ln, 4, axis=1).ravel()
    cols = np.tile(ln, (1, 4)).ravel()
    key = np.unique(rows * n + cols)
    r, c = key // n, key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp), c


def _positions(row_ptr, cols, rows, want):
    """Position of column want[k] inside row rows[k] of a CSR pattern (columns
    ascending): one search over (row, column) keys."""
    rows = np.asarray(rows, dtype=np.int64)
    want = np.asarray(want, dtype=np.int64)
    if rows.size == 0:
        return np.zeros(0, dtype=np.int64)
    n = int(row_ptr.size - 1)
    big = max(int(cols.max(initial=0)), int(want.max(initial=0))) + 1
    keyed = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr)) * big + cols
    q = rows * big + want
    out = np.searchsorted(keyed, q)
    if np.any(out >= keyed.size) or np.any(keyed[np.minimum(out, keyed.size - 1)] != q):
        raise ValueError("entry not in the pattern")
    return out


@dataclass
class RankPlan:
    """What rank ``rank`` of ``world`` assembles, owns and exchanges."""

    rank: int
    world: int
    elems: np.ndarray        # int64 [E_r] global element ids
    nodes: np.ndarray        # int64 [n_r] global ids of the nodes those elements touch (ascending)
    lnods: np.ndarray        # int32 [E_r, 4] local node ids
    coord: np.ndarray        # float64 [n_r, 3]
    own_rows: np.ndarray     # int64 [n_own] global ids of the owned nodes (ascending)
    own_row_ptr: np.ndarray  # int64 [n_own + 1] global pattern of the owned rows
    own_cols: np.ndarray     # int64 [nnz_own] global column ids
    local_row_ptr: np.ndarray  # int64 [n_r + 1] pattern of the local assembly (local ids)
    local_cols: np.ndarray     # int64
    keep_src: np.ndarray = field(default=None)  # local CSR positions of entries of owned rows
    keep_dst: np.ndarray = field(default=None)  # their positions in the owned pattern
    keep_node_src: np.ndarray = field(default=None)  # local node ids of owned nodes
    keep_node_dst: np.ndarray = field(default=None)  # their index among the owned rows
    send_src: list = field(default_factory=list)      # per peer: local CSR positions sent
    send_node_src: list = field(default_factory=list)  # per peer: local node ids sent (rhs)
    recv_dst: list = field(default_factory=list)      # per peer: owned-pattern positions received
    recv_node_dst: list = field(default_factory=list)  # per peer: owned-row indices received

    @property
    def n_own(self):
        return int(self.own_rows.size)

    @property
    def nnz_own(self):
        return int(self.own_cols.size)


def build_plans(coord, lnods, world: int, part=None):
    """RankPlan of every rank (host setup; every rank can build all of them
    from the global mesh, or only its own with ``build_plans(...)[rank]``)."""
    coord = np.asarray(coord, dtype=np.float64)
    lnods = np.asarray(lnods, dtype=np.int64)
    n = coord.shape[0]
    part = rcb_partition(coord, lnods, world) if part is None else np.asarray(part)
    # owner: the lowest rank touching the node
    owner = np.full(n, world, dtype=np.int64)
    for r in range(world):
        touched = np.unique(lnods[part == r])
        owner[touched] = np.minimum(owner[touched], r)
    g_rp, g_cols = _pattern(n, lnods)
    plans = []
    for r in range(world):
        el = np.flatnonzero(part == r)
        nodes = np.unique(lnods[el]) if el.size else np.zeros(0, dtype=np.int64)
        loc = np.full(n, -1, dtype=np.int64)
        loc[nodes] = np.arange(nodes.size)
        ln_loc = loc[lnods[el]].astype(np.int32) if el.size else np.zeros((0, 4), dtype=np.int32)
        l_rp, l_cols = _pattern(nodes.size, ln_loc)
        own = np.flatnonzero(owner == r)
        o_rp = np.concatenate([[0], np.cumsum(g_rp[own + 1] - g_rp[own])]).astype(np.int64)
        o_cols = np.concatenate([g_cols[g_rp[i]:g_rp[i + 1]] for i in own]) if own.size else np.zeros(0, np.int64)
        plans.append(RankPlan(rank=r, world=world, elems=el, nodes=nodes, lnods=ln_loc, coord=coord[nodes],
                              own_rows=own, own_row_ptr=o_rp, own_cols=o_cols, local_row_ptr=l_rp, local_cols=l_cols))
    # routing: every local entry (row i, col j) and node value goes to the
    # owner of node i (kept when that is the rank itself)
    own_index = np.full(n, -1, dtype=np.int64)
    for p in plans:
        own_index[p.own_rows] = np.arange(p.n_own)
    empty = np.zeros(0, dtype=np.int32)
    for p in plans:
        p.send_src, p.send_node_src = [empty] * world, [empty] * world
        p.recv_dst, p.recv_node_dst = [empty] * world, [empty] * world
    for p in plans:
        lrows = np.repeat(np.arange(p.nodes.size), np.diff(p.local_row_ptr))
        g_rows, g_cols_e = p.nodes[lrows], p.nodes[p.local_cols]
        dest, node_dest = owner[g_rows], owner[p.nodes]
        for s in range(world):
            q = plans[s]
            sel = np.flatnonzero(dest == s)
            pos = _positions(q.own_row_ptr, q.own_cols, own_index[g_rows[sel]], g_cols_e[sel]).astype(np.int32)
            nsel = np.flatnonzero(node_dest == s)
            nidx = own_index[p.nodes[nsel]].astype(np.int32)
            if s == p.rank:
                p.keep_src, p.keep_dst = sel.astype(np.int32), pos
                p.keep_node_src, p.keep_node_dst = nsel.astype(np.int32), nidx
            else:
                p.send_src[s], p.send_node_src[s] = sel.astype(np.int32), nsel.astype(np.int32)
                q.recv_dst[p.rank], q.recv_node_dst[p.rank] = pos, nidx
    return plans


def exchange(send: list, recv_counts: list, group=None):
    """All-to-all of per-peer value blocks: send[s] (a tensor, [count_s, c])
    goes to rank s; returns the blocks received from every rank (rank order).
    One torch.distributed all_to_all_single over the flattened buffers."""
    import torch
    import torch.distributed as dist

    c = send[0].shape[1] if send and send[0].dim() == 2 else 1
    flat = torch.cat([t.reshape(-1, c) for t in send]).contiguous()
    out = torch.empty((int(sum(recv_counts)), c), dtype=flat.dtype, device=flat.device)
    in_split = [int(t.shape[0]) for t in send]
    dist.all_to_all_single(out, flat, output_split_sizes=[int(x) for x in recv_counts],
                           input_split_sizes=in_split, group=group)
    return list(torch.split(out, [int(x) for x in recv_counts]))


class PartitionedAssembler:
    """Rank ``plan.rank``'s share of one mesh on its GPU (see the module text).

    ``assemble(u_local)`` takes the velocities of the rank's nodes
    (``plan.nodes`` order, [3, n_r]) and returns (A [nnz_own], G [3, nnz_own],
    rhs [3, n_own]) of the rows the rank owns, after the exchange;
    ``assemble_stabilized(u_local)`` does the same for the stabilised velocity
    block (Auu [9, nnz_own], G, rhs: twelve values per interface entry
    instead of four).  With ``exchange_fn`` another transport than
    torch.distributed can move the blocks (the single-GPU test passes the
    blocks between the ranks of one process)."""

    def __init__(self, plan: RankPlan, precision="mixed64", device=None):
        import torch

        from . import Assembler

        self.plan = plan
        self.asm = Assembler(plan.coord, plan.lnods, precision=precision, device=device)
        rp, ci = (t.cpu().numpy() for t in self.asm.pattern())
        if not (np.array_equal(rp, plan.local_row_ptr) and np.array_equal(ci, plan.local_cols)):
            raise ValueError("the library's local CSR pattern differs from the plan's")
        dev = self.asm.device if isinstance(self.asm.device, torch.device) else torch.device("cuda", self.asm.device)
        idx = lambda a: torch.as_tensor(np.asarray(a, dtype=np.int32), device=dev)  # noqa: E731
        self.keep_src, self.keep_dst = idx(plan.keep_src), idx(plan.keep_dst)
        self.keep_node_src, self.keep_node_dst = idx(plan.keep_node_src), idx(plan.keep_node_dst)
        self.send_src = [idx(a) for a in plan.send_src]
        self.send_node_src = [idx(a) for a in plan.send_node_src]
        self.recv_dst = [idx(a) for a in plan.recv_dst]
        self.recv_node_dst = [idx(a) for a in plan.recv_node_dst]
        self.dtype = self.asm.out_dtype
        self.dev = dev

    @staticmethod
    def _chunks(A, G):
        """The entry-value arrays in chunks of at most four components (what
        one nsi_gather_values / nsi_add_values call moves), as (first, rest,
        count): (A, G_x, G_y, G_z) for the assembly; (Auu 0-3), (Auu 4-7),
        (Auu 8, G_x, G_y, G_z) for the stabilised block."""
        if A.dim() == 1:
            return [(A, G, 4)]
        return [(None, A[0:4], 4), (None, A[4:8], 4), (A[8], G, 4)]

    def _gather(self, chunks, stride, idx):
        import torch

        from . import gather_values

        parts = [gather_values(f, r, stride, idx, nc) for f, r, nc in chunks]
        return parts[0] if len(parts) == 1 else torch.cat(parts, dim=1)

    @staticmethod
    def _add(chunks, stride, idx, vals):
        from . import add_values

        c0 = 0
        for f, r, nc in chunks:
            add_values(f, r, stride, idx, vals[:, c0:c0 + nc], nc)
            c0 += nc

    def local(self, u_local, rho=1.0, mu=1e-3, dt=1e-2):
        """Step 1: the local assembly."""
        return self.asm.assemble(u_local, rho=rho, mu=mu, dt=dt)

    def local_stabilized(self, u_local, rho=1.0, mu=1e-3, dt=1e-2):
        """Step 1 for the stabilised velocity block."""
        return self.asm.assemble_stabilized(u_local, rho=rho, mu=mu, dt=dt)

    def pack(self, A, G, rhs):
        """Step 2: per peer, the entries [count, c] (A, G_x, G_y, G_z; or the
        nine Auu components, then G) and node values [count, 3] of rows that
        peer owns."""
        from . import gather_values

        chunks = self._chunks(A, G)
        ent = [self._gather(chunks, self.plan.local_cols.size, s) for s in self.send_src]
        nod = [gather_values(None, rhs, self.plan.nodes.size, s, ncomp=3) for s in self.send_node_src]
        return ent, nod

    def finish(self, A, G, rhs, recv_ent, recv_nod):
        """Step 4: the owned rows -- own entries, then each peer's in rank order."""
        import torch

        from . import add_values, gather_values

        p = self.plan
        oA = torch.zeros((p.nnz_own,) if A.dim() == 1 else (A.shape[0], p.nnz_own), dtype=self.dtype,
                         device=self.dev)
        oG = torch.zeros(3, p.nnz_own, dtype=self.dtype, device=self.dev)
        orhs = torch.zeros(3, p.n_own, dtype=self.dtype, device=self.dev)
        own = self._chunks(oA, oG)
        self._add(own, p.nnz_own, self.keep_dst, self._gather(self._chunks(A, G), p.local_cols.size, self.keep_src))
        own_nod = gather_values(None, rhs, p.nodes.size, self.keep_node_src, ncomp=3)
        add_values(None, orhs, p.n_own, self.keep_node_dst, own_nod, ncomp=3)
        for s in range(p.world):
            if s == p.rank:
                continue
            self._add(own, p.nnz_own, self.recv_dst[s], recv_ent[s])
            add_values(None, orhs, p.n_own, self.recv_node_dst[s], recv_nod[s], ncomp=3)
        return oA, oG, orhs

    def _exchange_and_finish(self, A, G, rhs, exchange_fn, group):
        ent, nod = self.pack(A, G, rhs)
        p = self.plan
        counts_ent = [int(x.size) for x in p.recv_dst]
        counts_nod = [int(x.size) for x in p.recv_node_dst]
        if exchange_fn is None:
            recv_ent = exchange(ent, counts_ent, group)
            recv_nod = exchange(nod, counts_nod, group)
        else:
            recv_ent, recv_nod = exchange_fn(ent, nod)
        return self.finish(A, G, rhs, recv_ent, recv_nod)

    def assemble(self, u_local, rho=1.0, mu=1e-3, dt=1e-2, exchange_fn=None, group=None):
        A, G, rhs = self.local(u_local, rho, mu, dt)
        return self._exchange_and_finish(A, G, rhs, exchange_fn, group)

    def assemble_stabilized(self, u_local, rho=1.0, mu=1e-3, dt=1e-2, exchange_fn=None, group=None):
        Auu, G, rhs = self.local_stabilized(u_local, rho, mu, dt)
        return self._exchange_and_finish(Auu, G, rhs, exchange_fn, group)

    def close(self):
        self.asm.close()
