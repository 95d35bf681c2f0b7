"""Block partition across ranks (one GPU each) and the cross-rank halo.

Host-side planning for the multi-device form of the solver:

* Cartesian splitting of every parent block into child blocks (Section 4:
  a 3D/2D decomposition that cuts the most non-contiguous index direction
  first - k, then j, then i - into near-equal slabs), with the number of
  children per parent proportional to its cells and an optional
  over-decomposition factor;
* aggregation of the children onto ranks (Section 4's "domain aggregation"
  for np not much larger than the number of parent blocks): largest child
  first onto the least-loaded rank;
* decomposition and re-linking of the parent blocks' connected boundaries
  and physical boundary patches onto the children (Section 5), and new
  connections across every cut;
* per rank: its blocks as a problem of their own (connections with both
  sides on the rank stay ordinary connections, exchanged on the device by
  the library's exchange kernel), and its halo tables - the connections
  whose other side lives on another rank - for fv_set_halo, ordered so that
  each sender's and receiver's segments for one another match item for item.

The transfer (``TorchTransport``) posts every receive and send of a rank
before it waits on any of them (Section 7.2 V5/V6): no rank blocks on one
boundary while a neighbour blocks on another, so the circular wait of
Section 5 cannot arise, and no boundary reordering is needed.  Device
buffers go to NCCL directly (V10, GPUDirect); host buffers to gloo.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np

GHOST = 2


@dataclass
class Child:
    """A child block: cells [lo, lo + n) of parent block ``parent`` (per axis
    i, j, k) on rank ``rank``."""
    parent: int
    lo: Tuple[int, int, int]
    n: Tuple[int, int, int]
    rank: int = 0

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def _tangential(axis: int) -> Tuple[int, int]:
    """Tangential axes of a face normal to ``axis``, in (i, j, k) order."""
    return tuple(a for a in range(3) if a != axis)


def _cuts(ext: int, parts: int) -> List[int]:
    """Near-equal cut positions 0 = x_0 < ... < x_parts = ext."""
    return [(t * ext) // parts for t in range(parts + 1)]


def split_counts(ext: Sequence[int], n: int, dim: int, min_ext: int = 4) -> Tuple[int, int, int]:
    """Parts (p_i, p_j, p_k) with p_i p_j p_k = n that keep every child at
    least ``min_ext`` cells thick along a cut axis and minimise the cut area;
    among equal areas the one cutting k most, then j (Section 4 decomposes
    the most non-contiguous direction first).  None if no split of n works."""
    best = None
    for pk in range(1, n + 1):
        if n % pk or (dim == 2 and pk > 1):
            continue
        for pj in range(1, n // pk + 1):
            if (n // pk) % pj:
                continue
            pi = n // (pk * pj)
            p = (pi, pj, pk)
            if any(p[a] > 1 and ext[a] // p[a] < min_ext for a in range(3)):
                continue
            area = sum((p[a] - 1) * ext[_tangential(a)[0]] * ext[_tangential(a)[1]] for a in range(3))
            key = (area, -pk, -pj)
            if best is None or key < best[0]:
                best = (key, p)
    return None if best is None else best[1]


@dataclass
class Partition:
    """Children of every parent block, their ranks, and the connections and
    boundary patches re-linked onto them (child indices are global)."""
    children: List[Child]
    conns: list
    bcs: list
    nranks: int
    dim: int

    # -- bookkeeping ----------------------------------------------------------
    def rank_children(self, r: int) -> List[int]:
        """Global child indices on rank r, in ascending order (their local
        numbering on that rank)."""
        return [c for c, ch in enumerate(self.children) if ch.rank == r]

    def loads(self) -> List[int]:
        out = [0] * self.nranks
        for ch in self.children:
            out[ch.rank] += ch.ncells
        return out

    def imbalance(self) -> float:
        """max rank load / mean rank load (1 = perfectly balanced)."""
        ld = self.loads()
        return max(ld) / (sum(ld) / len(ld))

    # -- rank-local problem ------------------------------------------------------
    def local_problem(self, pb, r: int):
        """The blocks of rank r as a problem of their own: geometry, state
        (with the parent's ghost values where a child touches a parent
        boundary), source, boundary patches and the connections with both
        sides on rank r, in local numbering.  Connections to other ranks are
        the halo tables (``halo``)."""
        sub = self.problem_of(pb, self.rank_children(r))
        sub.name = "%s_rank%d_of_%d" % (pb.name, r, self.nranks)
        return sub

    def problem_of(self, pb, mine: Sequence[int]):
        """Children ``mine`` (global indices, in their local order) as one
        problem, with the connections and patches among them."""
        import cases
        loc = {g: n for n, g in enumerate(mine)}
        parents = cases.unpack_state(pb.blocks, pb.q)
        blocks, states, src = [], [], [] if pb.source is not None else None
        for g in mine:
            ch = self.children[g]
            P = pb.blocks[ch.parent]
            (i0, j0, k0), (ni, nj, nk) = ch.lo, ch.n
            if P.nodes is not None:
                nodes = np.ascontiguousarray(P.nodes[k0:k0 + nk + 1, j0:j0 + nj + 1, i0:i0 + ni + 1])
                b = cases.BlockDesc(ni, nj, nk, nodes)
            else:
                x0 = tuple(P.x0[a] + ch.lo[a] * P.h[a] for a in range(3))
                b = cases.BlockDesc(ni, nj, nk, None, x0, tuple(P.h))
            blocks.append(b)
            qg = parents[ch.parent]
            states.append(np.ascontiguousarray(qg[:, k0:k0 + nk + 2 * GHOST, j0:j0 + nj + 2 * GHOST,
                                                  i0:i0 + ni + 2 * GHOST]))
            if src is not None:
                src.append(np.ascontiguousarray(pb.source[ch.parent][:, k0:k0 + nk, j0:j0 + nj, i0:i0 + ni]))
        conns = []
        for c in self.conns:
            if c.dst_block in loc and c.src_block in loc:
                conns.append(cases.Connection(loc[c.dst_block], c.dst_face, tuple(c.dst_lo), tuple(c.dst_hi),
                                              loc[c.src_block], c.src_face, tuple(c.src_lo), tuple(c.transform)))
        bcs = [cases.BCPatch(loc[p.block], p.face, tuple(p.lo), tuple(p.hi), p.kind, tuple(p.state))
               for p in self.bcs if p.block in loc]
        return cases.Problem(blocks, conns, pb.dim, cases.pack_state(blocks, states), src, pb.dt, dict(pb.params),
                             pb.name, bcs)

    def halo(self, r: int):
        """Halo tables of rank r: (send, recv, send_ranges, recv_ranges).
        send / recv are connections in rank r's local numbering (the remote
        side's block index -1) for fv_set_halo; *_ranges map a peer rank to
        the (offset, length) in doubles of its segment of the send / receive
        buffer.  Segments run over peers in ascending order; inside one, the
        connections in global order - the same order on both sides."""
        import cases
        loc = {g: n for n, g in enumerate(self.rank_children(r))}
        send, recv = [], []
        send_ranges: Dict[int, Tuple[int, int]] = {}
        recv_ranges: Dict[int, Tuple[int, int]] = {}
        soff = roff = 0
        for peer in range(self.nranks):
            if peer == r:
                continue
            s0, r0 = soff, roff
            for c in self.conns:
                d_rank = self.children[c.dst_block].rank
                s_rank = self.children[c.src_block].rank
                cells = 5 * 2 * (c.dst_hi[0] - c.dst_lo[0]) * (c.dst_hi[1] - c.dst_lo[1])
                if s_rank == r and d_rank == peer:
                    send.append(cases.Connection(-1, c.dst_face, tuple(c.dst_lo), tuple(c.dst_hi),
                                                 loc[c.src_block], c.src_face, tuple(c.src_lo), tuple(c.transform)))
                    soff += cells
                if d_rank == r and s_rank == peer:
                    recv.append(cases.Connection(loc[c.dst_block], c.dst_face, tuple(c.dst_lo), tuple(c.dst_hi),
                                                 -1, c.src_face, tuple(c.src_lo), tuple(c.transform)))
                    roff += cells
            if soff > s0:
                send_ranges[peer] = (s0, soff - s0)
            if roff > r0:
                recv_ranges[peer] = (r0, roff - r0)
        return send, recv, send_ranges, recv_ranges


def partition(pb, nranks: int, over: float = 1.0, min_ext: int = 4) -> Partition:
    """Split the blocks of problem ``pb`` and aggregate them onto ``nranks``
    ranks (Section 4), then decompose and re-link its connections and
    boundary patches onto the children (Section 5).

    Each parent gets n_b = max(1, round(cells_b / W)) children with W = total
    cells / (nranks * over) (more children when fewer than nranks result);
    n_b is lowered until a split with children at least ``min_ext`` cells
    thick along every cut axis exists.  Children go to ranks largest first,
    each onto the least-loaded rank (lowest index on ties)."""
    import cases
    if nranks < 1:
        raise ValueError("nranks must be at least 1")
    dim = pb.dim
    total = sum(b.ncells for b in pb.blocks)
    W = total / (nranks * over)
    counts = [max(1, int(round(b.ncells / W))) for b in pb.blocks]
    while sum(counts) < nranks:
        # more pieces where the current pieces are largest
        b = max(range(len(counts)), key=lambda x: (pb.blocks[x].ncells / counts[x], -x))
        counts[b] += 1
    splits = []
    for b, P in enumerate(pb.blocks):
        ext = (P.ni, P.nj, P.nk)
        n = counts[b]
        while True:
            p = split_counts(ext, n, dim, min_ext)
            if p is not None:
                break
            n -= 1
        splits.append(p)
    children: List[Child] = []
    first = []                      # first child index of each parent
    grid = []                       # per parent: cut positions per axis
    for b, P in enumerate(pb.blocks):
        ext = (P.ni, P.nj, P.nk)
        cuts = [_cuts(ext[a], splits[b][a]) for a in range(3)]
        grid.append(cuts)
        first.append(len(children))
        for kk in range(splits[b][2]):
            for jj in range(splits[b][1]):
                for ii in range(splits[b][0]):
                    idx = (ii, jj, kk)
                    lo = tuple(cuts[a][idx[a]] for a in range(3))
                    n = tuple(cuts[a][idx[a] + 1] - cuts[a][idx[a]] for a in range(3))
                    children.append(Child(b, lo, n))
    # aggregation onto ranks: largest first, least-loaded rank
    load = [0] * nranks
    for c in sorted(range(len(children)), key=lambda x: (-children[x].ncells, x)):
        r = min(range(nranks), key=lambda x: (load[x], x))
        children[c].rank = r
        load[r] += children[c].ncells

    def child_at(b: int, cell: Sequence[int]) -> int:
        """Child of parent b holding parent cell index ``cell`` (i, j, k)."""
        idx = [int(np.searchsorted(grid[b][a], cell[a], side="right")) - 1 for a in range(3)]
        return first[b] + (idx[2] * splits[b][1] + idx[1]) * splits[b][0] + idx[0]

    def face_children(b: int, face: int) -> List[int]:
        """Children of parent b whose face ``face`` lies on the parent's."""
        a = face // 2
        P = pb.blocks[b]
        ext = (P.ni, P.nj, P.nk)
        out = []
        for c in range(first[b], first[b] + splits[b][0] * splits[b][1] * splits[b][2]):
            ch = children[c]
            on = ch.lo[a] == 0 if face % 2 == 0 else ch.lo[a] + ch.n[a] == ext[a]
            if on:
                out.append(c)
        return out

    conns = []
    # 1. new connections across every cut (identity orientation)
    for b in range(len(pb.blocks)):
        for c in range(first[b], first[b] + splits[b][0] * splits[b][1] * splits[b][2]):
            A = children[c]
            for a in range(3):
                if A.lo[a] + A.n[a] == (pb.blocks[b].ni, pb.blocks[b].nj, pb.blocks[b].nk)[a]:
                    continue
                cell = list(A.lo)
                cell[a] = A.lo[a] + A.n[a]
                Bc = child_at(b, cell)
                t0, t1 = _tangential(a)
                full = (A.n[t0], A.n[t1])
                # B's min-face ghosts <- A's cells at its max face, and back
                conns.append(cases.Connection(Bc, 2 * a, (0, 0), full, c, 2 * a + 1, (0, 0), (1, 2)))
                conns.append(cases.Connection(c, 2 * a + 1, (0, 0), full, Bc, 2 * a, (0, 0), (1, 2)))
    # 2. the parents' connections, decomposed over dst and src children
    for pc in pb.conns:
        da, sa = pc.dst_face // 2, pc.src_face // 2
        dt = _tangential(da)
        stt = _tangential(sa)
        T = tuple(pc.transform)
        u = [abs(T[0]) - 1, abs(T[1]) - 1]
        sg = [1 if T[0] > 0 else -1, 1 if T[1] > 0 else -1]

        def to_src(x0: int, x1: int):
            """src parent tangential coordinates (per src tangential axis,
            in order) of dst parent tangential coordinates (x0, x1)."""
            st = [pc.src_lo[0], pc.src_lo[1]]
            st[u[0]] += sg[0] * (x0 - pc.dst_lo[0])
            st[u[1]] += sg[1] * (x1 - pc.dst_lo[1])
            return st

        for D in face_children(pc.dst_block, pc.dst_face):
            Dc = children[D]
            lo0 = max(pc.dst_lo[0], Dc.lo[dt[0]])
            hi0 = min(pc.dst_hi[0], Dc.lo[dt[0]] + Dc.n[dt[0]])
            lo1 = max(pc.dst_lo[1], Dc.lo[dt[1]])
            hi1 = min(pc.dst_hi[1], Dc.lo[dt[1]] + Dc.n[dt[1]])
            if lo0 >= hi0 or lo1 >= hi1:
                continue
            for S in face_children(pc.src_block, pc.src_face):
                Sc = children[S]
                # dst range along each dst tangential axis t whose image lies
                # in S along src tangential axis u[t]
                rng = []
                for t, (lo, hi) in enumerate(((lo0, hi0), (lo1, hi1))):
                    s_lo = Sc.lo[stt[u[t]]]
                    s_hi = s_lo + Sc.n[stt[u[t]]]
                    # image of x: src_lo[u] + sg (x - dst_lo[t]) in [s_lo, s_hi)
                    if sg[t] > 0:
                        a = pc.dst_lo[t] + (s_lo - pc.src_lo[u[t]])
                        bnd = pc.dst_lo[t] + (s_hi - pc.src_lo[u[t]])
                    else:
                        a = pc.dst_lo[t] - (s_hi - 1 - pc.src_lo[u[t]])
                        bnd = pc.dst_lo[t] - (s_lo - 1 - pc.src_lo[u[t]])
                    rng.append((max(lo, a), min(hi, bnd)))
                (q0, e0), (q1, e1) = rng
                if q0 >= e0 or q1 >= e1:
                    continue
                st = to_src(q0, q1)
                conns.append(cases.Connection(
                    D, pc.dst_face, (q0 - Dc.lo[dt[0]], q1 - Dc.lo[dt[1]]),
                    (e0 - Dc.lo[dt[0]], e1 - Dc.lo[dt[1]]),
                    S, pc.src_face, (st[0] - Sc.lo[stt[0]], st[1] - Sc.lo[stt[1]]), T))
    # 3. physical boundary patches
    bcs = []
    for p in getattr(pb, "bcs", []) or []:
        t = _tangential(p.face // 2)
        for D in face_children(p.block, p.face):
            Dc = children[D]
            lo = [max(p.lo[x], Dc.lo[t[x]]) for x in range(2)]
            hi = [min(p.hi[x], Dc.lo[t[x]] + Dc.n[t[x]]) for x in range(2)]
            if lo[0] < hi[0] and lo[1] < hi[1]:
                bcs.append(cases.BCPatch(D, p.face, (lo[0] - Dc.lo[t[0]], lo[1] - Dc.lo[t[1]]),
                                         (hi[0] - Dc.lo[t[0]], hi[1] - Dc.lo[t[1]]), p.kind, tuple(p.state)))
    return Partition(children, conns, bcs, nranks, dim)


def split_problem(pb, part: Partition):
    """All children of ``part`` as one problem (every re-linked connection an
    ordinary one): the serial counterpart of the partitioned run, the
    paper's parallel-vs-serial comparison."""
    sub = part.problem_of(pb, list(range(len(part.children))))
    sub.name = pb.name + "_split%d" % len(part.children)
    return sub


def gather_interior(pb, part: Partition, rank_states: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Parent interiors (5, nk, nj, ni) assembled from every rank's packed
    ghosted state (in rank order)."""
    import cases
    out = [np.zeros((5, b.nk, b.nj, b.ni)) for b in pb.blocks]
    for r, q in enumerate(rank_states):
        mine = part.rank_children(r)
        blocks = [cases.BlockDesc(*part.children[g].n) for g in mine]
        for g, qb, b in zip(mine, cases.unpack_state(blocks, q), blocks):
            ch = part.children[g]
            (i0, j0, k0), (ni, nj, nk) = ch.lo, ch.n
            out[ch.parent][:, k0:k0 + nk, j0:j0 + nj, i0:i0 + ni] = cases.interior_view(b, qb)
    return out


# ---------------------------------------------------------------------------
# transfer and the partitioned RK stage
# ---------------------------------------------------------------------------

class TorchTransport:
    """Halo transfer over torch.distributed point-to-point calls: every
    receive and every send of this rank is posted (one message per peer and
    direction) before any is waited on (Section 7.2 V5/V6).  Device buffers
    go through NCCL, host buffers through gloo."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, ranks) -> None:
        import torch.distributed as dist
        (rs,) = ranks                     # one rank per process
        ops = []
        for peer, (o, n) in sorted(rs.recv_ranges.items()):
            ops.append(dist.P2POp(dist.irecv, rs.recv_buf[o:o + n], peer, self.group))
        for peer, (o, n) in sorted(rs.send_ranges.items()):
            ops.append(dist.P2POp(dist.isend, rs.send_buf[o:o + n], peer, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


class LoopbackTransport:
    """All ranks in one process (tests; no rank waits on another): each
    receiver's segment from a peer is a device copy of that peer's segment
    for it."""

    def exchange(self, ranks) -> None:
        by_rank = {rs.rank: rs for rs in ranks}
        for rs in ranks:
            for peer, (o, n) in rs.recv_ranges.items():
                so, sn = by_rank[peer].send_ranges[rs.rank]
                assert sn == n, "halo segments of ranks %d -> %d differ" % (peer, rs.rank)
                rs.recv_buf[o:o + n].copy_(by_rank[peer].send_buf[so:so + sn])


class RankSolver:
    """One rank's share of a partitioned problem: a library handle for its
    blocks (their mutual connections exchanged on the device) with the halo
    tables of its cross-rank connections, and device send/receive buffers."""

    def __init__(self, pb, part: Partition, rank: int, precision: str = "fp64", **kw):
        import torch
        from ._binding import Solver
        if pb.params.get("visc", 0):
            # a halo slab carries state values only: the viscous terms' ghost
            # geometry and depth-1 edge ghosts at a cross-rank cut would not
            # be the donor's, so the partitioned form is inviscid
            raise ValueError("the partitioned form covers the inviscid residual (visc = 0)")
        self.rank = rank
        self.problem = part.local_problem(pb, rank)
        self.solver = Solver.from_problem(self.problem, precision=precision, **kw)
        send, recv, self.send_ranges, self.recv_ranges = part.halo(rank)
        self.solver.set_halo(send, recv)
        self.send_buf = torch.zeros(max(1, self.solver.halo_size(False)), dtype=torch.float64, device="cuda")
        self.recv_buf = torch.zeros(max(1, self.solver.halo_size(True)), dtype=torch.float64, device="cuda")
        self.n_stages = self.solver.n_stages

    def set_state(self, q=None):
        import torch
        q = self.problem.q if q is None else q
        self.solver.set_state(torch.from_numpy(q).cuda() if isinstance(q, np.ndarray) else q)
        if self.problem.source is not None:
            self.solver.set_source(torch.from_numpy(
                np.concatenate([x.ravel() for x in self.problem.source])).cuda())

    def close(self):
        self.solver.close()


def exchange_halos(ranks: Sequence[RankSolver], buffer: int, transport) -> None:
    """Pack every rank's send slabs of state buffer ``buffer``, transfer,
    unpack into the ghosts (the ranks' own connections and boundaries are
    filled by the library's stage call)."""
    for rs in ranks:
        rs.solver.halo_pack(buffer, rs.send_buf)
    transport.exchange(ranks)
    for rs in ranks:
        rs.solver.halo_unpack(buffer, rs.recv_buf)


def rk_stage(ranks: Sequence[RankSolver], m: int, dt: float, transport) -> None:
    """RK stage m on every rank: halo of the stage input, then the library's
    stage (own connections, boundaries, fused residual + update)."""
    b_in = ranks[0].solver.stage_buffers(m)[0]
    exchange_halos(ranks, b_in, transport)
    for rs in ranks:
        rs.solver.rk_stage(m, dt)


def rk_step(ranks: Sequence[RankSolver], dt: float, transport) -> None:
    for m in range(1, ranks[0].n_stages + 1):
        rk_stage(ranks, m, dt, transport)


def residual(ranks: Sequence[RankSolver], transport, buffer: int = 0):
    """Residual of every rank's blocks after the full ghost fill."""
    exchange_halos(ranks, buffer, transport)
    out = []
    for rs in ranks:
        rs.solver.exchange_ghosts(buffer)
        out.append(rs.solver.residual(buffer))
    return out
