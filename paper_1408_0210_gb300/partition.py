"""Multi-GPU split of the EIFMM evaluation (host logic).

Two splits, both free of TMA multicast and of any kernel that waits on
another GPU:

* Right-hand-side columns.  Many sigma vectors sharing one tree (the paper's
  many-query setting, Section 1) split by columns: every rank holds the
  whole tree and operator set and evaluates its own columns; nothing is
  exchanged during the evaluation.  `rhs_columns` gives a rank's range and
  `evaluate_rhs_sharded` runs it.

* Space.  The leaves, in Morton order, split into contiguous ranges aligned
  to the subtrees of a partition level m (the boxes of level m own whole
  subtrees).  For its leaves a rank needs (Algorithm 3 and Section 3.2):
    - the points and sigma of the halo leaves, the neighbours of its leaves
      that it does not own (the near field f_N);
    - at every level k > m, the multipole coefficients What of the boxes in
      the interaction lists of its boxes that it does not own (step 4);
    - the levels 2..m whole: every rank forms the What of its own level-m
      boxes, the ranks all-gather them, and the levels above m are formed
      redundantly on every rank.
  `spatial_plan` computes these sets; `exchange_plan` turns them into what
  each rank sends to each other rank.

Box indices are Morton keys at their level (x bit lowest), as everywhere in
the library.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# right-hand-side columns
# --------------------------------------------------------------------------
def rhs_columns(n_rhs: int, world_size: int, rank: int) -> tuple[int, int]:
    """Contiguous column range [c0, c1) of `rank`: the columns split as evenly
    as possible, the first n_rhs % world_size ranks taking one more."""
    if not (0 <= rank < world_size) or n_rhs < 0:
        raise ValueError("rank outside [0, world_size) or negative n_rhs")
    q, r = divmod(n_rhs, world_size)
    c0 = rank * q + min(rank, r)
    return c0, c0 + q + (1 if rank < r else 0)


def evaluate_rhs_sharded(tree, ops, sigma, f, prec, rank: int, world_size: int, stream=None) -> tuple[int, int]:
    """Evaluates this rank's columns of sigma (n_src, R) into the same columns
    of f (n_tgt, R) (column-major CUDA tensors); returns the column range.
    No communication: each rank owns its columns of f."""
    from . import eifmm as E
    c0, c1 = rhs_columns(sigma.shape[1], world_size, rank)
    if c1 > c0:
        E.eifmm_evaluate(tree, ops, sigma[:, c0:c1], f[:, c0:c1], prec, stream)
    return c0, c1


# --------------------------------------------------------------------------
# space
# --------------------------------------------------------------------------
def morton_coords(keys: np.ndarray, level: int) -> np.ndarray:
    """(n, 3) integer box coordinates of Morton keys at `level`."""
    keys = np.asarray(keys, dtype=np.int64)
    c = np.zeros((keys.size, 3), dtype=np.int64)
    for b in range(level):
        for a in range(3):
            c[:, a] |= ((keys >> (3 * b + a)) & 1) << b
    return c


def morton_keys_of(c: np.ndarray, level: int) -> np.ndarray:
    """Morton keys of (n, 3) integer box coordinates at `level`."""
    c = np.asarray(c, dtype=np.int64)
    k = np.zeros(c.shape[0], dtype=np.int64)
    for b in range(level):
        for a in range(3):
            k |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return k


def leaf_ranges(leaf_counts: np.ndarray, depth: int, m: int, world_size: int) -> list[tuple[int, int]]:
    """Split the 8^depth leaves into world_size contiguous Morton ranges made
    of whole level-m subtrees (8^(depth - m) leaves each), balanced by point
    count: rank r takes the subtrees whose cumulative count starts in
    [r W / N, (r + 1) W / N), W the total count.  Returns [(a, b)] leaf
    ranges; a rank may own none (a == b) when there are fewer subtrees than
    ranks."""
    if not (1 <= m <= depth):
        raise ValueError("partition level m must lie in [1, depth]")
    cnt = np.asarray(leaf_counts, dtype=np.int64)
    if cnt.size != 8 ** depth:
        raise ValueError("leaf_counts needs 8^depth entries")
    sub = 8 ** (depth - m)
    per = cnt.reshape(8 ** m, sub).sum(axis=1)
    start = np.concatenate([[0], np.cumsum(per)[:-1]])
    total = max(int(per.sum()), 1)
    owner = np.minimum((start * world_size) // total, world_size - 1)
    owner = np.maximum.accumulate(owner)  # monotone: contiguous ranges
    out = []
    for r in range(world_size):
        idx = np.nonzero(owner == r)[0]
        if idx.size == 0:
            # an empty range placed where the owners move past r
            j = int(np.searchsorted(owner, r))
            out.append((j * sub, j * sub))
        else:
            out.append((int(idx[0]) * sub, (int(idx[-1]) + 1) * sub))
    return out


_NBR = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], dtype=np.int64)
_FAR = np.array([(dx, dy, dz) for dz in range(-3, 4) for dy in range(-3, 4) for dx in range(-3, 4)
                 if max(abs(dx), abs(dy), abs(dz)) > 1], dtype=np.int64)  # the 316 far offsets


def _shifted(keys: np.ndarray, level: int, offsets: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Every (box, offset) pair: the shifted box keys and whether they lie in
    the cube."""
    c = morton_coords(keys, level)
    s = c[:, None, :] + offsets[None, :, :]
    n = 1 << level
    ok = np.all((s >= 0) & (s < n), axis=2)
    return s, ok


def halo_leaves(a: int, b: int, depth: int, nonempty: np.ndarray | None = None) -> np.ndarray:
    """Leaves outside [a, b) adjacent to a leaf of [a, b) (the 27-leaf
    neighbourhood of Section 3.2), sorted; with `nonempty` (bool per leaf)
    only the owned leaves that hold points ask, and only halo leaves that
    hold points are kept."""
    own = np.arange(a, b, dtype=np.int64)
    if nonempty is not None:
        own = own[np.asarray(nonempty, dtype=bool)[own]]
    if own.size == 0:
        return np.zeros(0, dtype=np.int64)
    s, ok = _shifted(own, depth, _NBR)
    k = morton_keys_of(s[ok], depth)
    k = np.unique(k[(k < a) | (k >= b)])
    if nonempty is not None:
        k = k[np.asarray(nonempty, dtype=bool)[k]]
    return k


def interaction_list(level: int, box: int) -> np.ndarray:
    """Interaction list of `box` at `level` (Section 3.2): the children of
    the parent's neighbours that are not neighbours of the box, sorted."""
    c = morton_coords(np.array([box]), level)[0]
    n = 1 << level
    pc = c // 2
    lo = np.maximum(2 * (pc - 1), 0)
    hi = np.minimum(2 * (pc + 1) + 1, n - 1)
    out = []
    for z in range(lo[2], hi[2] + 1):
        for y in range(lo[1], hi[1] + 1):
            for x in range(lo[0], hi[0] + 1):
                if max(abs(x - c[0]), abs(y - c[1]), abs(z - c[2])) > 1:
                    out.append((x, y, z))
    return np.sort(morton_keys_of(np.array(out, dtype=np.int64).reshape(-1, 3), level))


def remote_boxes(a: int, b: int, depth: int, level: int) -> np.ndarray:
    """At `level` (> the partition level), the boxes outside the rank's
    subtrees that lie in the interaction list of one of its boxes: the What
    it must receive for step 4.  [a, b) is the rank's leaf range."""
    sh = 3 * (depth - level)
    a_k, b_k = a >> sh, b >> sh  # the rank's boxes at this level (whole subtrees)
    own = np.arange(a_k, b_k, dtype=np.int64)
    if own.size == 0:
        return np.zeros(0, dtype=np.int64)
    # I(I) lies within the 7^3 offsets of the parent's neighbourhood
    c = morton_coords(own, level)
    n = 1 << level
    pc = c // 2
    out = []
    for d in _FAR:
        s = c + d
        ok = np.all((s >= 0) & (s < n), axis=1)
        # in the interaction list: the parent of I + d neighbours the parent of I
        ok &= np.all(np.abs(s // 2 - pc) <= 1, axis=1)
        out.append(morton_keys_of(s[ok], level))
    k = np.unique(np.concatenate(out)) if out else np.zeros(0, dtype=np.int64)
    return k[(k < a_k) | (k >= b_k)]


def spatial_plan(leaf_counts: np.ndarray, depth: int, m: int, world_size: int, rank: int) -> dict:
    """What `rank` owns and needs: its leaf range, the halo leaves of its
    near field (non-empty ones), the remote boxes per level k = m + 1..depth
    whose What it receives, and the replicated levels 2..m."""
    ranges = leaf_ranges(leaf_counts, depth, m, world_size)
    a, b = ranges[rank]
    nonempty = np.asarray(leaf_counts) > 0
    return {"ranges": ranges, "leaves": (a, b), "partition_level": m,
            "halo": halo_leaves(a, b, depth, nonempty),
            "remote": {k: remote_boxes(a, b, depth, k) for k in range(m + 1, depth + 1)},
            "replicated_levels": list(range(2, m + 1))}


def owner_of(keys: np.ndarray, level: int, depth: int, ranges: list[tuple[int, int]]) -> np.ndarray:
    """Rank owning each box (Morton key at `level`) under the leaf ranges."""
    starts = np.array([r[0] for r in ranges], dtype=np.int64)
    ends = np.array([r[1] for r in ranges], dtype=np.int64)
    leaf = np.asarray(keys, dtype=np.int64) << (3 * (depth - level))
    own = np.searchsorted(starts, leaf, side="right") - 1
    # skip empty ranges that share a start with the next one
    for i in range(own.size):
        while ends[own[i]] <= leaf[i]:
            own[i] += 1
    return own


def exchange_plan(plans: list[dict], depth: int) -> dict:
    """From every rank's spatial plan, the messages of one evaluation:
    sends[(src, dst)] = {"halo": leaves whose points and sigma src sends to
    dst, k: boxes of level k whose What src sends to dst}."""
    ranges = plans[0]["ranges"]
    sends = {}
    for dst, p in enumerate(plans):
        own = owner_of(p["halo"], depth, depth, ranges)
        for src in np.unique(own):
            sends.setdefault((int(src), dst), {})["halo"] = p["halo"][own == src]
        for k, boxes in p["remote"].items():
            own = owner_of(boxes, k, depth, ranges)
            for src in np.unique(own):
                sends.setdefault((int(src), dst), {})[k] = boxes[own == src]
    return sends
