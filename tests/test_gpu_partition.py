"""One mesh split over ranks by element partition, each rank's share on the
library (local row-gather assembly, nsi_gather_values, nsi_add_values): the
ranks run here in one process on the one GPU, the exchange passing the packed
blocks between them directly (no kernel waits for another rank's), and the
owned rows of every rank must match the oracle's assembly of the whole mesh
and the library's single-mesh assembly within the precision's bar."""
import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")
from paper_2111_05651_gb300 import partition as pt  # noqa: E402

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_assembly_matches_whole_mesh(precision, world):
    mesh, u = meshgen.config_mesh(N=10, jitter=0.15, numbering="random", seed=96)
    plans = pt.build_plans(mesh.coord, mesh.lnods, world)
    ranks = [pt.PartitionedAssembler(p, precision=precision) for p in plans]
    local, packs = [], []
    for r, p in zip(ranks, plans):
        out = r.local(torch.as_tensor(u[p.nodes].T.copy()), RHO, MU, DT)
        local.append(out)
        packs.append(r.pack(*out))
    results = []
    for s, r in enumerate(ranks):  # rank s receives block s of every other rank's packs
        recv_ent = [packs[q][0][s] for q in range(world)]
        recv_nod = [packs[q][1][s] for q in range(world)]
        results.append(r.finish(*local[s], recv_ent, recv_nod))
    torch.cuda.synchronize()
    whole = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    wA, wG, wrhs = (t.double().cpu().numpy() for t in whole.assemble(torch.as_tensor(u.T.copy()), rho=RHO, mu=MU,
                                                                      dt=DT))
    wrp = whole.pattern()[0].cpu().numpy()
    whole.close()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    g_rp, g_ci, gA, gG, grhs = oracle.assemble(mesh.coord, mesh.lnods, uo, None, RHO, MU, DT)
    assert np.array_equal(wrp, g_rp)
    tol = TOL[precision]
    for p, (oA, oG, orhs) in zip(plans, results):
        oA, oG, orhs = oA.double().cpu().numpy(), oG.double().cpu().numpy(), orhs.double().cpu().numpy()
        for k, i in enumerate(p.own_rows):
            sl, ol = slice(g_rp[i], g_rp[i + 1]), slice(p.own_row_ptr[k], p.own_row_ptr[k + 1])
            for got, ref, lib in ((oA[ol], gA[sl], wA[sl]),) + tuple((oG[d, ol], gG[d, sl], wG[d, sl]) for d in range(3)):
                scale = max(np.abs(ref).max(), 1e-300)
                assert np.abs(got - ref).max() <= tol * scale
                assert np.abs(got - lib).max() <= 2 * tol * scale
        assert np.abs(orhs - grhs[:, p.own_rows]).max() <= tol * np.abs(grhs).max()
    for r in ranks:
        r.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_stabilized_block_matches_whole_mesh(precision, world):
    """The stabilised velocity block over ranks (twelve values per interface
    entry: the nine Auu components, then G): the owned rows of every rank
    against the oracle's stabilised assembly of the whole mesh and the
    library's single-mesh call, component by component."""
    mesh, u = meshgen.config_mesh(N=8, jitter=0.15, numbering="random", seed=97)
    plans = pt.build_plans(mesh.coord, mesh.lnods, world)
    ranks = [pt.PartitionedAssembler(p, precision=precision) for p in plans]
    local, packs = [], []
    for r, p in zip(ranks, plans):
        out = r.local_stabilized(torch.as_tensor(u[p.nodes].T.copy()), RHO, MU, DT)
        local.append(out)
        packs.append(r.pack(*out))
    assert all(e.shape[1] == 12 for e in packs[0][0])
    results = []
    for s, r in enumerate(ranks):
        recv_ent = [packs[q][0][s] for q in range(world)]
        recv_nod = [packs[q][1][s] for q in range(world)]
        results.append(r.finish(*local[s], recv_ent, recv_nod))
    torch.cuda.synchronize()
    whole = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    wAuu, wG, wrhs = (t.double().cpu().numpy()
                      for t in whole.assemble_stabilized(torch.as_tensor(u.T.copy()), rho=RHO, mu=MU, dt=DT))
    whole.close()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    g_rp, g_ci, gAuu, gG, grhs = oracle.assemble_stabilized(mesh.coord, mesh.lnods, uo, None, RHO, MU, DT)
    tol = TOL[precision]
    for p, (oAuu, oG, orhs) in zip(plans, results):
        oAuu, oG, orhs = oAuu.double().cpu().numpy(), oG.double().cpu().numpy(), orhs.double().cpu().numpy()
        assert oAuu.shape == (9, p.nnz_own)
        for k, i in enumerate(p.own_rows):
            sl, ol = slice(g_rp[i], g_rp[i + 1]), slice(p.own_row_ptr[k], p.own_row_ptr[k + 1])
            pairs = tuple((oAuu[c, ol], gAuu[c, sl], wAuu[c, sl]) for c in range(9)) + \
                tuple((oG[d, ol], gG[d, sl], wG[d, sl]) for d in range(3))
            for got, ref, lib in pairs:
                scale = max(np.abs(ref).max(), 1e-300)
                assert np.abs(got - ref).max() <= tol * scale
                assert np.abs(got - lib).max() <= 2 * tol * scale
        assert np.abs(orhs - grhs[:, p.own_rows]).max() <= tol * np.abs(grhs).max()
    for r in ranks:
        r.close()
