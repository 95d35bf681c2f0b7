"""Block partition and cross-rank halo (host side, no GPU).

* The children tile every parent block exactly once, every cut leaves
  children at least 4 cells thick, every rank gets work, and the load is
  balanced (Section 4's splitting and aggregation).
* The paper's parallel-vs-serial check (Section 8 compares the partitioned
  and serial solutions to 1e-12): the CPU oracle run on all children with
  the re-linked connections (Section 5) reproduces the oracle run on the
  parent blocks bit for bit - residual and RK stages - for a curvilinear
  block with fixed ghosts, a periodic block, seeded blocks with rotated and
  flipped connections, and the 2D inlet with physical boundaries.
* Two gloo ranks, each stepping its own children with the oracle, exchange
  their halo slabs through the package's transport (every send and receive
  posted before the wait) and again reproduce the serial run bit for bit.
  The slab items are gathered and scattered here from the connection
  definition (cases.Connection), independently of the CUDA kernels that do
  it on the device.
"""
import os

import numpy as np
import pytest

import cases
import oracle
from paper_2012_02925_gb300 import partition as P


def _problems():
    yield "mms", cases.mms_3d((20, 14, 12), curvilinear=True)
    yield "periodic", cases.large_periodic(24, 20, 16, nbumps=3)
    yield "multiblock", cases.multiblock_batched(nblocks=5, lo=8, hi=18, seed=3)
    yield "inlet", cases.inlet_2d(52, 16)


@pytest.mark.parametrize("nranks,over", [(2, 1.0), (3, 1.0), (5, 2.0), (8, 1.0)])
def test_children_tile_every_parent(nranks, over):
    for name, pb in _problems():
        part = P.partition(pb, nranks, over=over)
        for b, blk in enumerate(pb.blocks):
            cover = np.zeros((blk.nk, blk.nj, blk.ni), dtype=np.int32)
            for ch in part.children:
                if ch.parent != b:
                    continue
                (i0, j0, k0), (ni, nj, nk) = ch.lo, ch.n
                cover[k0:k0 + nk, j0:j0 + nj, i0:i0 + ni] += 1
                ext = (blk.ni, blk.nj, blk.nk)
                for a in range(3):
                    if ch.n[a] != ext[a]:
                        assert ch.n[a] >= 4, (name, ch)
            assert (cover == 1).all(), name
        if len(part.children) >= nranks:
            assert min(part.loads()) > 0, name
        assert sum(part.loads()) == pb.ncells


def test_load_balance_of_the_seeded_batch():
    """64 uneven blocks (10.9 M cells) on 8 ranks: aggregation keeps the
    most loaded rank within 10 % of the mean."""
    pb = cases.multiblock_batched()
    part = P.partition(pb, 8)
    assert part.imbalance() < 1.10
    part = P.partition(pb, 8, over=2.0)
    assert part.imbalance() < 1.05


def _serial_and_split(pb, nranks, over, nstages):
    part = P.partition(pb, nranks, over=over)
    sp = P.split_problem(pb, part)
    o, os_ = oracle.Oracle(pb), oracle.Oracle(sp)
    q, qs = o.fill_ghosts(pb.q.copy()), os_.fill_ghosts(sp.q.copy())
    return part, sp, (o, q), (os_, qs)


@pytest.mark.parametrize("nranks,over", [(2, 1.0), (3, 1.0), (4, 2.0)])
def test_split_problem_reproduces_the_serial_oracle_bit_for_bit(nranks, over):
    for name, pb in _problems():
        part, sp, (o, q), (os_, qs) = _serial_and_split(pb, nranks, over, 8)
        r = o.residual(q)
        rs = os_.residual(qs)
        # child residuals back into the parents' layout
        R = [r[o.roffs[n]:o.roffs[n + 1]].reshape(5, b.nk, b.nj, b.ni) for n, b in enumerate(pb.blocks)]
        for g, ch in enumerate(part.children):
            (i0, j0, k0), (ni, nj, nk) = ch.lo, ch.n
            got = rs[os_.roffs[g]:os_.roffs[g + 1]].reshape(5, nk, nj, ni)
            assert np.array_equal(got, R[ch.parent][:, k0:k0 + nk, j0:j0 + nj, i0:i0 + ni]), name
        ref = o.run(pb.q.copy(), pb.dt, 8)
        got = os_.run(sp.q.copy(), pb.dt, 8)
        ref_i = [cases.interior_view(b, x) for b, x in zip(pb.blocks, cases.unpack_state(pb.blocks, ref))]
        whole = P.Partition(part.children, part.conns, part.bcs, 1, part.dim)
        for ch in whole.children:
            ch.rank = 0
        got_i = P.gather_interior(pb, whole, [got])
        for a, b in zip(got_i, ref_i):
            assert np.array_equal(a, b), name


def test_a_wrong_relink_is_caught():
    """Planted mistake: the ghosts across one cut taken from the wrong
    neighbour (a child of the same size elsewhere in the block) change the
    split run, so the bit-for-bit comparison above can fail."""
    pb = cases.large_periodic(24, 20, 16, nbumps=3)
    part = P.partition(pb, 3)
    c = part.conns[0]
    wrong = next(g for g in range(len(part.children)) if g not in (c.src_block, c.dst_block))
    part.conns[0] = cases.Connection(c.dst_block, c.dst_face, c.dst_lo, c.dst_hi, wrong, c.src_face,
                                     c.src_lo, c.transform)
    sp = P.split_problem(pb, part)
    o, os_ = oracle.Oracle(pb), oracle.Oracle(sp)
    ref = o.run(pb.q.copy(), pb.dt, 4)
    got = os_.run(sp.q.copy(), pb.dt, 4)
    whole = P.Partition(part.children, part.conns, part.bcs, 1, part.dim)
    for ch in whole.children:
        ch.rank = 0
    got_i = P.gather_interior(pb, whole, [got])[0]
    ref_i = cases.interior_view(pb.blocks[0], cases.unpack_state(pb.blocks, ref)[0])
    assert not np.array_equal(got_i, ref_i)


# ---------------------------------------------------------------------------
# two gloo ranks
# ---------------------------------------------------------------------------

def _tangential(a):
    return [x for x in range(3) if x != a]


def slab_cells(conn, blk, side):
    """Flat indices, in one variable plane of a block's ghosted state, of a
    slab's items in the order (a, b, depth), a fastest: the donor cells of a
    sender's connection (side "src", blk = its src block) or the ghost cells
    of a receiver's (side "dst", blk = its dst block), from the connection's
    definition."""
    L0, L1 = conn.dst_hi[0] - conn.dst_lo[0], conn.dst_hi[1] - conn.dst_lo[1]
    ext = (blk.ni, blk.nj, blk.nk)
    shape = (blk.nk + 4, blk.nj + 4, blk.ni + 4)
    out = []
    for d in (1, 2):
        for b in range(L1):
            for a in range(L0):
                c = [0, 0, 0]
                if side == "dst":
                    da = conn.dst_face // 2
                    t = _tangential(da)
                    c[t[0]], c[t[1]] = conn.dst_lo[0] + a, conn.dst_lo[1] + b
                    c[da] = ext[da] - 1 + d if conn.dst_face % 2 else -d
                else:
                    sa = conn.src_face // 2
                    s = _tangential(sa)
                    st = [conn.src_lo[0], conn.src_lo[1]]
                    for tt, step in ((conn.transform[0], a), (conn.transform[1], b)):
                        st[abs(tt) - 1] += step if tt > 0 else -step
                    c[s[0]], c[s[1]] = st
                    c[sa] = ext[sa] - d if conn.src_face % 2 else d - 1
                out.append(np.ravel_multi_index((c[2] + 2, c[1] + 2, c[0] + 2), shape))
    return np.array(out)


class _HostRank:
    """A rank's halo buffers as CPU tensors, for TorchTransport over gloo."""

    def __init__(self, rank, sub, send, recv, send_ranges, recv_ranges):
        import torch
        self.rank, self.sub = rank, sub
        self.send, self.recv = send, recv
        self.send_ranges, self.recv_ranges = send_ranges, recv_ranges
        ns = sum(5 * 2 * (c.dst_hi[0] - c.dst_lo[0]) * (c.dst_hi[1] - c.dst_lo[1]) for c in send)
        nr = sum(5 * 2 * (c.dst_hi[0] - c.dst_lo[0]) * (c.dst_hi[1] - c.dst_lo[1]) for c in recv)
        self.send_buf = torch.zeros(max(1, ns), dtype=torch.float64)
        self.recv_buf = torch.zeros(max(1, nr), dtype=torch.float64)
        self.offs = cases.core.block_offsets(sub.blocks)

    def _plane(self, q, blk, v):
        n = cases.core.ghosted_cells(self.sub.blocks[blk])
        return q[self.offs[blk] + v * n: self.offs[blk] + (v + 1) * n]

    def pack(self, q):
        buf = self.send_buf.numpy()
        o = 0
        for c in self.send:
            donors = slab_cells(c, self.sub.blocks[c.src_block], "src")
            n = len(donors)
            for v in range(5):
                buf[o + v * n:o + (v + 1) * n] = self._plane(q, c.src_block, v)[donors]
            o += 5 * n

    def unpack(self, q):
        buf = self.recv_buf.numpy()
        o = 0
        for c in self.recv:
            ghosts = slab_cells(c, self.sub.blocks[c.dst_block], "dst")
            n = len(ghosts)
            for v in range(5):
                self._plane(q, c.dst_block, v)[ghosts] = buf[o + v * n:o + (v + 1) * n]
            o += 5 * n


def _gloo_rank(rank, world, port, name, nstages, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = dict(_problems())[name]
    part = P.partition(pb, world, over=2.0)
    sub = part.local_problem(pb, rank)
    send, recv, sr, rr = part.halo(rank)
    hr = _HostRank(rank, sub, send, recv, sr, rr)
    tr = P.TorchTransport()
    o = oracle.Oracle(sub, threads=1)
    M = o.M
    cur = sub.q.copy()
    q0 = cur
    for s in range(nstages):
        m = s % M + 1
        if m == 1:
            q0 = cur
        hr.pack(cur)
        tr.exchange([hr])
        qin = cur.copy()
        hr.unpack(qin)
        cur = o.rk_stage(q0, qin, m, pb.dt)
    states = [None] * world
    dist.all_gather_object(states, cur)
    if rank == 0:
        out["interior"] = P.gather_interior(pb, part, states)
        out["halo"] = (len(send), len(recv))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["multiblock", "periodic"])
def test_two_gloo_ranks_reproduce_the_serial_run(name):
    import torch.multiprocessing as mp
    pb = dict(_problems())[name]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29600 + os.getpid() % 1000 + (7 if name == "periodic" else 0)
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, name, 8, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert out["halo"][0] > 0 and out["halo"][1] > 0
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 8)
    ref_i = [cases.interior_view(b, x) for b, x in zip(pb.blocks, cases.unpack_state(pb.blocks, ref))]
    for a, b in zip(out["interior"], ref_i):
        assert np.array_equal(a, b)


def test_rank_solver_refuses_viscous_problems():
    """A halo slab carries state values only, not the viscous terms' ghost
    geometry or edge ghosts, so the partitioned form refuses visc = 1
    before touching a GPU."""
    pb = cases.mms_3d(12, curvilinear=True, visc=1, mu=0.05)
    part = P.partition(pb, 2)
    with pytest.raises(ValueError):
        P.RankSolver(pb, part, 0)
