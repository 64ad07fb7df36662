"""The multi-GPU split of the evaluation (host logic), on CPU.

Right-hand-side columns: the ranges of all ranks tile the columns.  Space:
two gloo ranks each compute their plan (leaf range, halo leaves, remote
boxes per level, replicated levels) and exchange it; every set is checked
against a brute-force list built from the CPU checker's own neighbour and
interaction lists (Section 3.2), and the messages of the exchange plan
against what the receiving rank needs."""
import os
import socket

import numpy as np
import pytest

from paper_1408_0210_gb300 import partition as PT
from paper_1408_0210_gb300 import workloads as wl

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def test_rhs_columns_tile_the_columns():
    for R in (0, 1, 7, 64):
        for ws in (1, 2, 3, 8):
            cols = [PT.rhs_columns(R, ws, r) for r in range(ws)]
            assert cols[0][0] == 0 and cols[-1][1] == R
            assert all(cols[i][1] == cols[i + 1][0] for i in range(ws - 1))
            sizes = [c1 - c0 for c0, c1 in cols]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        PT.rhs_columns(8, 2, 2)


def test_interaction_list_matches_checker(orc):
    rng = np.random.default_rng(3)
    for level in (2, 3, 4):
        for box in rng.integers(0, 8 ** level, 40):
            np.testing.assert_array_equal(PT.interaction_list(level, int(box)),
                                          np.sort(orc.interaction_list(level, int(box))))


def _counts(n, depth, seed):
    x = wl.gaussian_mixture(n, seed)
    keys = np.zeros(n, dtype=np.int64)
    c = np.minimum((x * (1 << depth)).astype(np.int64), (1 << depth) - 1)
    for b in range(depth):
        for a in range(3):
            keys |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return np.bincount(keys, minlength=8 ** depth)


def _brute_halo(orc, a, b, depth, counts):
    out = set()
    for leaf in range(a, b):
        if counts[leaf] == 0:
            continue
        for nb in orc.neighbours(depth, leaf):
            if not (a <= nb < b) and counts[nb] > 0:
                out.add(int(nb))
    return np.array(sorted(out), dtype=np.int64)


def _brute_remote(orc, a, b, depth, level):
    sh = 3 * (depth - level)
    out = set()
    for box in range(a >> sh, b >> sh):
        for j in orc.interaction_list(level, box):
            if not ((a >> sh) <= j < (b >> sh)):
                out.add(int(j))
    return np.array(sorted(out), dtype=np.int64)


def _rank(rank, world, port, depth, m, counts, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = PT.spatial_plan(counts, depth, m, world, rank)
        plans = [None] * world
        dist.all_gather_object(plans, plan)
        sends = PT.exchange_plan(plans, depth)
        # what this rank sends, as it computes it, against what the others need
        mine = {dst: msg for (src, dst), msg in sends.items() if src == rank}
        out[rank] = (plan, mine, plans)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("depth,m", [(4, 1), (4, 2), (3, 1)])
def test_two_rank_spatial_plan_against_brute_force(orc, depth, m):
    counts = _counts(20000, depth, 7)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, depth, m, counts, out), nprocs=2, join=True)
        res = dict(out)
    plans = [res[0][0], res[1][0]]
    ranges = plans[0]["ranges"]
    # the ranges tile the leaves in order, in whole level-m subtrees
    assert ranges[0][0] == 0 and ranges[-1][1] == 8 ** depth and ranges[0][1] == ranges[1][0]
    assert all(r[0] % 8 ** (depth - m) == 0 for r in ranges)
    assert abs(int(counts[:ranges[0][1]].sum()) - int(counts[ranges[1][0]:].sum())) <= counts.sum() // 2
    for r, p in enumerate(plans):
        a, b = p["leaves"]
        np.testing.assert_array_equal(p["halo"], _brute_halo(orc, a, b, depth, counts))
        assert p["replicated_levels"] == list(range(2, m + 1))
        for k in range(m + 1, depth + 1):
            np.testing.assert_array_equal(p["remote"][k], _brute_remote(orc, a, b, depth, k))
    # rank 0 sends to rank 1 exactly what rank 1 needs and owns none of, and back
    for src, dst in ((0, 1), (1, 0)):
        msg = res[src][1].get(dst, {})
        np.testing.assert_array_equal(msg.get("halo", np.zeros(0, np.int64)), plans[dst]["halo"])
        a, b = plans[src]["leaves"]
        assert all(a <= x < b for x in msg.get("halo", []))
        for k in range(m + 1, depth + 1):
            np.testing.assert_array_equal(msg.get(k, np.zeros(0, np.int64)), plans[dst]["remote"][k])
