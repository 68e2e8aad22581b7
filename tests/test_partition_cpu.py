"""One mesh over several ranks (element partition + interface-row sum): the
host logic on CPU.  The plans (partition, ownership, routing of every local
entry) are checked for exact coverage; then world-size-2 and -3 gloo ranks
run the exchange of paper_2111_05651_gb300.partition with each rank's local
assembly computed by the FP64 oracle on its own elements (the GPU runs the
same plans with the library's kernels in test_gpu_partition.py), and every
owned row must equal the oracle's assembly of the whole mesh."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import meshgen
import oracle
from paper_2111_05651_gb300 import partition as pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


def _mesh():
    return meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=95)


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_partition_balanced_and_plans_cover_every_entry(world):
    mesh, _ = _mesh()
    part = pt.rcb_partition(mesh.coord, mesh.lnods, world)
    counts = np.bincount(part, minlength=world)
    assert counts.max() - counts.min() <= 1
    plans = pt.build_plans(mesh.coord, mesh.lnods, world, part)
    n = mesh.n_nodes
    g_rp, g_ci = oracle.pattern(n, mesh.lnods)
    owned = np.concatenate([p.own_rows for p in plans])
    assert np.array_equal(np.sort(owned), np.arange(n))  # every node owned once
    for p in plans:
        # the owned rows carry the global pattern
        for k, i in enumerate(p.own_rows):
            assert np.array_equal(p.own_cols[p.own_row_ptr[k]:p.own_row_ptr[k + 1]], g_ci[g_rp[i]:g_rp[i + 1]])
        # every local entry and node is kept or sent exactly once
        src = np.concatenate([p.keep_src] + [x for x in p.send_src])
        assert np.array_equal(np.sort(src), np.arange(p.local_cols.size))
        nsrc = np.concatenate([p.keep_node_src] + [x for x in p.send_node_src])
        assert np.array_equal(np.sort(nsrc), np.arange(p.nodes.size))
        for s, q in enumerate(plans):
            assert q.recv_dst[p.rank].size == p.send_src[s].size
            assert q.recv_node_dst[p.rank].size == p.send_node_src[s].size
    # every (owned row, column) receives at least one contribution
    for q in plans:
        hit = np.zeros(q.nnz_own, dtype=int)
        np.add.at(hit, q.keep_dst, 1)
        for s in range(world):
            np.add.at(hit, q.recv_dst[s], 1)
        assert hit.min() >= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q, stab=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh, u = _mesh()
        plan = pt.build_plans(mesh.coord, mesh.lnods, world)[rank]
        ul = u[plan.nodes]
        if stab:  # the stabilised block: nine Auu components per entry, then G
            _, _, A, G, rhs = oracle.assemble_stabilized(plan.coord, plan.lnods, ul, None, RHO, MU, DT)
        else:
            _, _, A, G, rhs = oracle.assemble(plan.coord, plan.lnods, ul, None, RHO, MU, DT)
        A = A.reshape(-1, A.shape[-1])  # [1 or 9, nnz]
        ent = [torch.as_tensor(np.c_[A[:, s_].T, G[:, s_].T]) for s_ in plan.send_src]  # [count, 4 or 12]
        nod = [torch.as_tensor(rhs[:, s_].T.copy()) for s_ in plan.send_node_src]  # [count, 3]
        recv_ent = pt.exchange(ent, [x.size for x in plan.recv_dst])
        recv_nod = pt.exchange(nod, [x.size for x in plan.recv_node_dst])
        c = A.shape[0]
        oA = np.zeros((c, plan.nnz_own)); oG = np.zeros((3, plan.nnz_own)); orhs = np.zeros((3, plan.n_own))
        oA[:, plan.keep_dst] += A[:, plan.keep_src]
        oG[:, plan.keep_dst] += G[:, plan.keep_src]
        orhs[:, plan.keep_node_dst] += rhs[:, plan.keep_node_src]
        for s in range(world):
            if s == rank:
                continue
            v, w = recv_ent[s].numpy(), recv_nod[s].numpy()
            oA[:, plan.recv_dst[s]] += v[:, :c].T
            oG[:, plan.recv_dst[s]] += v[:, c:].T
            orhs[:, plan.recv_node_dst[s]] += w.T
        q.put((rank, plan.own_rows, plan.own_row_ptr, oA, oG, orhs))
    finally:
        dist.destroy_process_group()


def _run_ranks(world, stab):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, stab)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _check_owned_rows(res, g_rp, gA, gG, grhs, n):
    seen = 0
    for rank, rows, rp, oA, oG, orhs in res:
        for k, i in enumerate(rows):
            sl = slice(g_rp[i], g_rp[i + 1])
            ol = slice(rp[k], rp[k + 1])
            for c in range(gA.shape[0]):
                scale = max(np.abs(gA[c, sl]).max(), 1e-300)
                assert np.abs(oA[c, ol] - gA[c, sl]).max() <= 1e-12 * scale
            for d in range(3):
                sg = max(np.abs(gG[d, sl]).max(), 1e-300)
                assert np.abs(oG[d, ol] - gG[d, sl]).max() <= 1e-12 * sg
        assert np.abs(orhs - grhs[:, rows]).max() <= 1e-12 * np.abs(grhs).max()
        seen += rows.size
    assert seen == n


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_exchange_gives_the_whole_mesh_assembly(world):
    res = _run_ranks(world, stab=False)
    mesh, u = _mesh()
    g_rp, g_ci, gA, gG, grhs = oracle.assemble(mesh.coord, mesh.lnods, u, None, RHO, MU, DT)
    _check_owned_rows(res, g_rp, gA[None, :], gG, grhs, mesh.n_nodes)


def test_gloo_exchange_gives_the_whole_mesh_stabilized_block():
    """The stabilised block over two gloo ranks: twelve values per interface
    entry (the nine Auu components, then G), the owned rows equal to the
    whole mesh's stabilised assembly."""
    res = _run_ranks(2, stab=True)
    mesh, u = _mesh()
    g_rp, g_ci, gAuu, gG, grhs = oracle.assemble_stabilized(mesh.coord, mesh.lnods, u, None, RHO, MU, DT)
    _check_owned_rows(res, g_rp, gAuu, gG, grhs, mesh.n_nodes)
