"""Octree node-descriptor builders (seeded input generation only).

A tree is a numpy int32 array of shape (n_nodes, 14) whose rows are
``level, ix, iy, iz, parent, child[8], tree_id``.  Rows are emitted breadth
first (root, then level 2, ...).  ``adaptive_tree`` enforces the nesting rule
that a node may only be refined when every same-level neighbour of it that
lies inside the domain exists.
"""

import itertools

import numpy as np

DESC_COLS = 14
N_SIDE = 8           # cells per sub-grid edge
N_CELLS = N_SIDE ** 3


def node_cell_width(level, box_size=1.0):
    """Cell width at ``level`` (root = level 1 holds 8 cells per edge)."""
    return box_size / (N_SIDE * 2 ** (level - 1))


def _neighbour_keys(level, ix, iy, iz):
    n = 2 ** (level - 1)
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        if dx == dy == dz == 0:
            continue
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        if 0 <= jx < n and 0 <= jy < n and 0 <= jz < n:
            yield (level, jx, jy, jz)


def _emit(refined, max_level, tree_id):
    """Build descriptor rows from per-level sets of refined node keys."""
    rows = []
    index = {}
    frontier = [(1, 0, 0, 0)]
    parent_of = {(1, 0, 0, 0): -1}
    for level in range(1, max_level + 1):
        nxt = []
        for key in sorted(frontier, key=lambda k: (k[3], k[2], k[1])):
            index[key] = len(rows)
            rows.append([key[0], key[1], key[2], key[3], parent_of[key]]
                        + [-1] * 8 + [tree_id])
        for key in sorted(frontier, key=lambda k: (k[3], k[2], k[1])):
            if key in refined.get(level, set()):
                _, ix, iy, iz = key
                for k in range(8):
                    ck = (level + 1, 2 * ix + (k & 1), 2 * iy + ((k >> 1) & 1),
                          2 * iz + ((k >> 2) & 1))
                    parent_of[ck] = index[key]
                    nxt.append(ck)
        frontier = nxt
        if not frontier:
            break
    # second pass: fill child indices (children were appended after parents)
    for key, i in index.items():
        level, ix, iy, iz = key
        for k in range(8):
            ck = (level + 1, 2 * ix + (k & 1), 2 * iy + ((k >> 1) & 1),
                  2 * iz + ((k >> 2) & 1))
            if ck in index:
                rows[i][5 + k] = index[ck]
    return np.asarray(rows, dtype=np.int32).reshape(-1, DESC_COLS)


def uniform_tree(max_level, tree_id=0):
    """Every node above ``max_level`` refined: 8**(max_level-1) leaf sub-grids."""
    refined = {}
    for level in range(1, max_level):
        n = 2 ** (level - 1)
        refined[level] = {(level, ix, iy, iz) for ix in range(n)
                          for iy in range(n) for iz in range(n)}
    return _emit(refined, max_level, tree_id)


def adaptive_tree(want_refine, max_level, box_lo=(0.0, 0.0, 0.0), box_size=1.0,
                  tree_id=0, min_level=1):
    """Refine nodes for which ``want_refine(lo, hi)`` is true, up to ``max_level``.

    ``lo``/``hi`` are the node's box corners.  Nodes above ``min_level`` are
    always refined.  Afterwards the refined sets are closed under the nesting
    rule (all in-domain same-level neighbours of a refined node must exist),
    working from the finest level upwards.
    """
    lo0 = np.asarray(box_lo, dtype=np.float64)
    refined = {}
    frontier = {(1, 0, 0, 0)}
    for level in range(1, max_level):
        width = box_size / 2 ** (level - 1)
        cur = set()
        for key in frontier:
            _, ix, iy, iz = key
            lo = lo0 + width * np.array([ix, iy, iz], dtype=np.float64)
            if level < min_level or want_refine(lo, lo + width):
                cur.add(key)
        refined[level] = cur
        frontier = set()
        for (_, ix, iy, iz) in cur:
            for k in range(8):
                frontier.add((level + 1, 2 * ix + (k & 1), 2 * iy + ((k >> 1) & 1),
                              2 * iz + ((k >> 2) & 1)))
    # closure, finest refined level first: a refined node needs its parent
    # refined (so that it exists) and every in-domain same-level neighbour to
    # exist (so their parents are refined).  Additions only go to coarser
    # levels, which are visited afterwards.
    for level in range(max_level - 1, 1, -1):
        for key in list(refined.get(level, ())):
            _, ix, iy, iz = key
            refined[level - 1].add((level - 1, ix // 2, iy // 2, iz // 2))
            for nb in _neighbour_keys(*key):
                _, jx, jy, jz = nb
                refined[level - 1].add((level - 1, jx // 2, jy // 2, jz // 2))
    return _emit(refined, max_level, tree_id)


def concat_trees(trees):
    """Stack several independent trees into one descriptor array."""
    out = []
    offset = 0
    for t_id, desc in enumerate(trees):
        d = desc.copy()
        d[:, 13] = t_id
        for col in range(4, 13):
            m = d[:, col] >= 0
            d[m, col] += offset
        out.append(d)
        offset += len(desc)
    return np.concatenate(out, axis=0)


def leaf_nodes(desc):
    """Indices of leaf nodes, in descriptor order (the order of density rows)."""
    return np.nonzero(desc[:, 5] < 0)[0]


def count_leaves(desc):
    return int((desc[:, 5] < 0).sum())


def leaf_cell_centres(desc, box_lo=(0.0, 0.0, 0.0), box_size=1.0):
    """Centres of all leaf cells, shape (n_leaf, 512, 3), cells x-fastest."""
    leaves = leaf_nodes(desc)
    lo = np.asarray(box_lo, dtype=np.float64)
    ar = np.arange(N_SIDE, dtype=np.float64)
    cz, cy, cx = np.meshgrid(ar, ar, ar, indexing="ij")
    local = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=-1)  # (512, 3)
    out = np.empty((len(leaves), N_CELLS, 3), dtype=np.float64)
    for j, i in enumerate(leaves):
        level, ix, iy, iz = (int(v) for v in desc[i, :4])
        h = node_cell_width(level, box_size)
        origin = np.array([ix, iy, iz], dtype=np.float64) * N_SIDE
        out[j] = lo + (origin + local + 0.5) * h
    return out
