"""Cross-rank halo on one GPU: the partitioned form (Sections 4-5, Section
7.2 V1/V5/V6) with its ranks as separate library handles in one process and
the transfer replaced by device copies (LoopbackTransport; no rank waits on
another).  fv_halo_pack / fv_halo_unpack move every cross-rank ghost cell, and
each handle exchanges its own connections, so the ranks together must
reproduce the single-handle run bit for bit: every face sees the same
operands and runs the same code.  The paper checks its parallel runs against
serial ones the same way (Section 8, 1e-12)."""
import numpy as np
import pytest

import cases
import oracle
from paper_2012_02925_gb300 import partition as P
from test_gpu_parity import rel_err_states, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROBLEMS = {
    "mms": lambda: cases.mms_3d((40, 19, 13), curvilinear=True),
    "periodic": lambda: cases.large_periodic(40, 24, 16, nbumps=3),
    "multiblock": lambda: cases.multiblock_batched(nblocks=8, lo=8, hi=24, seed=6),
    "inlet": lambda: cases.inlet_2d(104, 32),
}


def _ranks(pb, nranks, prec, over=1.0):
    part = P.partition(pb, nranks, over=over)
    ranks = [P.RankSolver(pb, part, r, precision=prec) for r in range(nranks)]
    for rs in ranks:
        rs.set_state()
    return part, ranks


def _gather(pb, part, ranks):
    states = [rs.solver.get_state(0).cpu().numpy() for rs in ranks]
    return P.gather_interior(pb, part, states)


def _interior(pb, q):
    return [cases.interior_view(b, x).copy() for b, x in zip(pb.blocks, cases.unpack_state(pb.blocks, q))]


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32flux"])
@pytest.mark.parametrize("name,nranks,over", [("mms", 2, 1.0), ("periodic", 3, 1.0), ("multiblock", 3, 2.0),
                                              ("inlet", 4, 1.0)])
def test_partitioned_ranks_reproduce_the_single_handle_run(prec, name, nranks, over):
    pb = PROBLEMS[name]()
    part, ranks = _ranks(pb, nranks, prec, over)
    tr = P.LoopbackTransport()
    assert any(rs.solver.halo_size(True) for rs in ranks)
    # residual after the full ghost fill
    rr = P.residual(ranks, tr)
    one = solver(pb, prec)
    one.exchange_ghosts(0)
    r1 = one.residual(0).cpu().numpy()
    o = oracle.Oracle(pb)
    R = [r1[o.roffs[n]:o.roffs[n + 1]].reshape(5, b.nk, b.nj, b.ni) for n, b in enumerate(pb.blocks)]
    for rs, r in zip(ranks, rr):
        r = r.cpu().numpy()
        ro = 0
        for g in part.rank_children(rs.rank):
            ch = part.children[g]
            (i0, j0, k0), (ni, nj, nk) = ch.lo, ch.n
            got = r[ro:ro + 5 * ni * nj * nk].reshape(5, nk, nj, ni)
            ro += 5 * ni * nj * nk
            assert np.array_equal(got, R[ch.parent][:, k0:k0 + nk, j0:j0 + nj, i0:i0 + ni])
    # two RK steps, graph-free (the halo runs between the library's stages)
    for rs in ranks:
        rs.set_state()
    for _ in range(2):
        P.rk_step(ranks, pb.dt, tr)
        one.rk_step(pb.dt, use_graph=False)
    got = _gather(pb, part, ranks)
    ref = _interior(pb, one.get_state(0).cpu().numpy())
    one.close()
    for rs in ranks:
        rs.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    if prec == "fp64":
        oref = o.run(pb.q.copy(), pb.dt, 8)
        for a, b in zip(got, _interior(pb, oref)):
            scale = np.abs(b).max(axis=(1, 2, 3))
            scale[1:4] = scale[1:4].max()
            assert (np.abs(a - b).max(axis=(1, 2, 3)) <= 1e-10 * scale).all()


def test_halo_tables_are_validated():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d((12, 10, 8), curvilinear=True)
    s = solver(pb, "fp64")
    # a receive patch outside the face
    bad = cases.Connection(0, 1, (0, 0), (11, 8), -1, 0, (0, 0), (1, 2))
    with pytest.raises(fv.FvError) as e:
        s.set_halo([], [bad])
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    # a send slab whose donors fall outside the src face
    bad = cases.Connection(-1, 0, (0, 0), (10, 8), 0, 1, (1, 0), (1, 2))
    with pytest.raises(fv.FvError) as e:
        s.set_halo([bad], [])
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    # two receive patches filling the same ghosts
    a = cases.Connection(0, 0, (0, 0), (6, 8), -1, 0, (0, 0), (1, 2))
    b = cases.Connection(0, 0, (5, 0), (10, 8), -1, 0, (0, 0), (1, 2))
    with pytest.raises(fv.FvError) as e:
        s.set_halo([], [a, b])
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s.set_halo([], [a])
    assert s.halo_size(True) == 5 * 2 * 6 * 8 and s.halo_size(False) == 0
    s.close()


def test_pack_then_unpack_is_the_exchange():
    """Pack of a slab on one handle, unpack of the same bytes on another:
    the ghosts equal the oracle's exchange bit for bit (a rotated connection
    between two blocks, split across two handles)."""
    pb = cases.rotated_split_problem(cases.mms_3d(12, curvilinear=True), 5)
    part = P.partition(pb, 1)
    part.children[1].rank = 1
    part.nranks = 2
    ranks = [P.RankSolver(pb, part, r, precision="fp64") for r in range(2)]
    rng = np.random.default_rng(2)
    q = pb.q + rng.normal(size=pb.q.shape) * 1e-3
    sub = [part.local_problem(cases.Problem(pb.blocks, pb.conns, pb.dim, q, pb.source, pb.dt, pb.params), r)
           for r in range(2)]
    for rs, sp in zip(ranks, sub):
        rs.solver.set_state(torch.from_numpy(sp.q).cuda())
    P.exchange_halos(ranks, 0, P.LoopbackTransport())
    for rs in ranks:
        rs.solver.exchange_ghosts(0)
    o = oracle.Oracle(pb)
    ref = cases.unpack_state(pb.blocks, o.exchange(q.copy()))
    for rs in ranks:
        got = rs.solver.get_state(0).cpu().numpy()
        (g,) = part.rank_children(rs.rank)
        assert np.array_equal(got.reshape(ref[g].shape), ref[g])
        rs.close()


def test_partitioned_full_size_batch():
    """The benchmark's 64-block batch (10.9 M cells, random orientations)
    on four ranks with over-decomposition: one RK step bit-equal to the
    single handle."""
    pb = cases.multiblock_batched()
    part, ranks = _ranks(pb, 4, "fp64", over=2.0)
    assert part.imbalance() < 1.05
    tr = P.LoopbackTransport()
    P.rk_step(ranks, pb.dt, tr)
    got = _gather(pb, part, ranks)
    for rs in ranks:
        rs.close()
    one = solver(pb, "fp64")
    one.rk_step(pb.dt, use_graph=False)
    ref = _interior(pb, one.get_state(0).cpu().numpy())
    one.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
