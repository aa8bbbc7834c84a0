"""The decomposition of one tree over several GPUs (fmm_partition, fmm_ghosts; the multi-node runs
of Sec. 5 split one tree), on the CPU: the partition's invariants, and two gloo ranks that each
evaluate the cells they own from their own leaves, the moments of the shared coarse cells summed
over the ranks (an all-reduce), and the densities and moments of the ghost subgrids the other
rank sends -- everything else they hold as NaN, so a ghost the list misses shows up as a NaN --
against the single-rank oracle solve; net force and torque summed over the ranks (an FP64
all-reduce) equal the whole solve's.  Not run on GPUs: this run has one GPU per box."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tree(levels):
    from paper_2101_08226_gb300 import api, synth
    w = synth.workload_binary(levels, axis=(1.0, 0.6, 0.3), offset=(0.02, -0.03, 0.05))
    return w, api.Tree(w.max_level, w.flags)


@pytest.mark.parametrize("n_ranks,cut", [(2, 2), (3, 2), (4, 3), (5, 1)])
def test_partition_invariants(n_ranks, cut):
    from paper_2101_08226_gb300 import synth
    w, t = _tree(4)
    rows = t.subgrids()
    owner = t.partition(n_ranks, cut)
    lev, leaf = rows[:, 0], rows[:, 4] == 1
    # shared: exactly the refined subgrids coarser than the cut
    assert np.array_equal(owner == -1, (lev < cut) & ~leaf)
    assert ((owner >= 0) & (owner < n_ranks))[owner != -1].all()
    # a subgrid below the cut has its parent's owner; Morton-contiguous runs at the cut level
    index = {tuple(r[:4]): k for k, r in enumerate(rows)}
    for k, r in enumerate(rows):
        if r[0] > cut:
            assert owner[k] == owner[index[(r[0] - 1, r[1] // 2, r[2] // 2, r[3] // 2)]]
    units = [k for k, r in enumerate(rows) if r[0] == cut or (r[0] < cut and r[4] == 1)]

    def key(k):
        l, i, j, kk = rows[k][:4]
        sh = cut - l
        i, j, kk = i << sh, j << sh, kk << sh
        m = 0
        for b in range(cut - 1, -1, -1):
            m = (m << 3) | (((i >> b) & 1) << 2) | (((j >> b) & 1) << 1) | ((kk >> b) & 1)
        return m
    ranks = [owner[k] for k in sorted(units, key=key)]
    assert ranks == sorted(ranks) and set(ranks) == set(range(n_ranks))
    # balance: every rank within one unit's weight of an equal share of the leaf cells
    n_leaf = leaf.sum() * 512
    per = np.array([(leaf & (owner == r)).sum() * 512 for r in range(n_ranks)])
    assert per.sum() == n_leaf
    below = {k: 0 for k in units}
    for k, r in enumerate(rows):
        if r[4] == 1:
            a = k
            l, i, j, kk = r[:4]
            while l > cut:
                l, i, j, kk = l - 1, i // 2, j // 2, kk // 2
            below[index[(l, i, j, kk)] if l == cut else k] += 512
    biggest = max(below.values())
    assert np.abs(per - n_leaf / n_ranks).max() <= biggest
    # ghosts: owned by another rank, never shared, sorted
    for r in range(n_ranks):
        gh = t.ghosts(owner, r)
        assert (owner[gh] != r).all() and (owner[gh] >= 0).all()
        assert np.array_equal(gh, np.unique(gh))


def _raw(mom):
    """(n, 40) centre-of-mass moments -> (n, 40) moments about the origin: m, m X, M2 + m X X,
    M3 + (M2 X, three placements) + m X X X (parallel axes)."""
    m = mom[:, 0]
    X = mom[:, 1:4]
    M2 = mom[:, 4:13].reshape(-1, 3, 3)
    M3 = mom[:, 13:40].reshape(-1, 3, 3, 3)
    R2 = M2 + m[:, None, None] * X[:, :, None] * X[:, None, :]
    R3 = (M3 + M2[:, :, :, None] * X[:, None, None, :] + M2[:, :, None, :] * X[:, None, :, None]
          + M2[:, None, :, :] * X[:, :, None, None]
          + m[:, None, None, None] * X[:, :, None, None] * X[:, None, :, None] * X[:, None, None, :])
    return np.concatenate([m[:, None], m[:, None] * X, R2.reshape(-1, 9), R3.reshape(-1, 27)], 1)


def _com(raw, centres):
    """Inverse of _raw; a cell without mass keeps its geometric centre and zero moments."""
    m = raw[:, 0]
    safe = np.where(m > 0, m, 1.0)
    X = np.where(m[:, None] > 0, raw[:, 1:4] / safe[:, None], centres)
    R2 = raw[:, 4:13].reshape(-1, 3, 3)
    R3 = raw[:, 13:40].reshape(-1, 3, 3, 3)
    M2 = R2 - m[:, None, None] * X[:, :, None] * X[:, None, :]
    M3 = (R3 - M2[:, :, :, None] * X[:, None, None, :] - M2[:, :, None, :] * X[:, None, :, None]
          - M2[:, None, :, :] * X[:, :, None, None]
          - m[:, None, None, None] * X[:, :, None, None] * X[:, None, :, None] * X[:, None, None, :])
    return np.concatenate([m[:, None], X, M2.reshape(-1, 9), M3.reshape(-1, 27)], 1)


def _rank_main(rank, world, port, levels, cut, out):
    import sys
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2101_08226_gb300 import synth
    w, t = _tree(levels)
    b = O.Tree(w.max_level, w.flags)
    rows = t.subgrids()
    leaf = rows[:, 4] == 1
    leaf_subs, inner_subs = np.nonzero(leaf)[0], np.nonzero(~leaf)[0]
    leaf_ord = {int(s): k for k, s in enumerate(leaf_subs)}
    inner_ord = {int(s): k for k, s in enumerate(inner_subs)}
    owner = t.partition(world, cut)
    ghosts = [t.ghosts(owner, r) for r in range(world)]
    rho_full = synth.leaf_density(w.field, b.leaves())
    # this rank's leaves only
    mine_leaf = np.repeat(owner[leaf_subs] == rank, 512)
    rho_mine = np.where(mine_leaf, rho_full, 0.0)
    mom_mine = O.inner_moments(b, rho_mine)          # moments of every refined cell from my leaves
    ctr = np.concatenate([synth.cell_centres(int(rows[s, 0]), rows[s, 1:4][None]) for s in inner_subs])
    # shared coarse cells: moments about the origin are additive over the ranks' leaves
    shared = np.repeat(owner[inner_subs] == -1, 512)
    raw = torch.from_numpy(np.ascontiguousarray(_raw(mom_mine[shared])))
    dist.all_reduce(raw, op=dist.ReduceOp.SUM)
    # ghosts: what every other rank needs from me
    send = {}
    for r in range(world):
        if r == rank:
            continue
        items = {}
        for s in ghosts[r]:
            s = int(s)
            if owner[s] != rank:
                continue
            if leaf[s]:
                items[s] = rho_full[leaf_ord[s] * 512:(leaf_ord[s] + 1) * 512].copy()
            else:
                items[s] = mom_mine[inner_ord[s] * 512:(inner_ord[s] + 1) * 512].copy()
        send[r] = items
    gathered = [None] * world
    dist.all_gather_object(gathered, send)
    # what this rank holds: its own data, the shared sums, the received ghosts; NaN elsewhere
    rho_loc = np.where(mine_leaf, rho_full, np.nan)
    mom_loc = np.full_like(mom_mine, np.nan)
    mine_inner = np.repeat(owner[inner_subs] == rank, 512)
    mom_loc[mine_inner] = mom_mine[mine_inner]
    mom_loc[shared] = _com(raw.numpy(), ctr[shared])
    for r in range(world):
        if r == rank:
            continue
        for s, data in gathered[r][rank].items():
            if leaf[s]:
                rho_loc[leaf_ord[s] * 512:(leaf_ord[s] + 1) * 512] = data
            else:
                mom_loc[inner_ord[s] * 512:(inner_ord[s] + 1) * 512] = data
    # evaluate: every cell of mine (small tree) or a sample with the cells next to other ranks
    my_cells = np.nonzero(mine_leaf)[0]
    if levels <= 3:
        idx = my_cells
    else:
        index = {tuple(int(v) for v in r[:4]): k for k, r in enumerate(rows)}
        nb_other = []
        for k, sg in enumerate(leaf_subs):
            if owner[sg] != rank:
                continue
            l, i, j, kk = (int(v) for v in rows[sg, :4])
            nbrs = [index.get((l, i + a, j + b_, kk + c)) for a in (-1, 0, 1) for b_ in (-1, 0, 1)
                    for c in (-1, 0, 1)]
            if any(q is not None and owner[q] not in (rank, -1) for q in nbrs):
                nb_other.append(k)
        rng = np.random.default_rng(rank)
        idx = np.unique(np.concatenate([rng.choice(my_cells, 200, replace=False)] +
                                       [k * 512 + rng.integers(0, 512, 4) for k in nb_other[:40]]))
    phi, g = O.sample_given(b, rho_loc, mom_loc, 0.5, idx)
    ps, gs = O.sample(b, rho_full, 0.5, idx)
    x, dx = synth.leaf_cell_centres(b.leaves())
    m = rho_full * dx ** 3
    f = m[idx, None] * g
    net = torch.tensor(np.concatenate([f.sum(0), np.cross(x[idx], f).sum(0)]))
    dist.all_reduce(net, op=dist.ReduceOp.SUM)
    out[rank] = {"finite": bool(np.isfinite(phi).all() and np.isfinite(g).all()),
                 "phi": float((np.abs(phi - ps) / np.abs(ps)).max()),
                 "g": float((np.linalg.norm(g - gs, axis=1) /
                             np.maximum(np.linalg.norm(gs, axis=1), 1e-6 * np.abs(gs).max())).max()),
                 "n_eval": int(idx.size), "n_ghost": int(len(ghosts[rank])),
                 "net": net.numpy().tolist(), "all_cells": levels <= 3}
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("levels,cut", [(3, 2), (4, 2)])
def test_two_ranks_with_exchanged_ghosts_equal_single_rank(levels, cut):
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), levels, cut, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r]["finite"], "a rank read data that neither it nor its ghosts hold"
        assert res[r]["phi"] <= 1e-11 and res[r]["g"] <= 1e-11, res[r]
        assert res[r]["n_ghost"] > 0 and res[r]["n_eval"] > 0
    if res[0]["all_cells"]:
        import oracle as O
        from paper_2101_08226_gb300 import synth
        w, t = _tree(levels)
        b = O.Tree(w.max_level, w.flags)
        rho = synth.leaf_density(w.field, b.leaves())
        _, g, _ = O.solve(b, rho, 0.5)
        x, dx = synth.leaf_cell_centres(b.leaves())
        f = (rho * dx ** 3)[:, None] * g
        ref = np.concatenate([f.sum(0), np.cross(x, f).sum(0)])
        S = (np.linalg.norm(x, axis=1) * np.linalg.norm(f, axis=1)).sum()
        net = np.asarray(res[0]["net"])
        assert np.abs(net - ref).max() <= 1e-13 * S
        assert np.abs(net).max() <= 1e-13 * S        # momentum and angular momentum conserved
