"""Pins of the oracle's greedy partition (Section 5.2, Algorithm 2) on graphs
whose good partitions are known: a square grid (blocks of four are 2 x 2
squares), a path numbered in any order (blocks are path segments), two
disconnected components (never mixed while one has l elements left), and the
tetrahedral box mesh (tile-external faces drop back to the native order's
level after a random renumbering)."""
import numpy as np
import pytest

import oracle
from oracle.partition import greedy_partition, partition_order
from workloads import kuhn_box_mesh


def grid_neighbours(n):
    nb = []
    for i in range(n):
        for j in range(n):
            nb.append([(i - 1) * n + j if i > 0 else -1, (i + 1) * n + j if i < n - 1 else -1,
                       i * n + j - 1 if j > 0 else -1, i * n + j + 1 if j < n - 1 else -1])
    return np.array(nb)


def path_neighbours(order):
    """Path visiting the labels in `order`; each label's two path neighbours."""
    K = len(order)
    nb = -np.ones((K, 4), dtype=np.int64)
    for p, e in enumerate(order):
        if p > 0:
            nb[e, 0] = order[p - 1]
        if p < K - 1:
            nb[e, 1] = order[p + 1]
    return nb


def check_partition(blocks, K, l):
    flat = [e for b in blocks for e in b]
    assert sorted(flat) == list(range(K))
    assert all(len(b) == l for b in blocks[:-1]) and 1 <= len(blocks[-1]) <= l


@pytest.mark.parametrize("n", [4, 6, 8])
def test_grid_blocks_of_four_are_squares(n):
    blocks = greedy_partition(grid_neighbours(n), 4)
    check_partition(blocks, n * n, 4)
    for b in blocks:
        rows, cols = {e // n for e in b}, {e % n for e in b}
        assert len(rows) == 2 and len(cols) == 2 and max(rows) - min(rows) == 1


def test_first_grid_block_in_queue_order():
    # seed 0; its neighbours 4 and 1 tie at one shared face, 4 was queued first
    assert greedy_partition(grid_neighbours(4), 4)[0] == [0, 4, 1, 5]


def test_next_block_seeded_by_the_first_queue_entry():
    """4 x 4 grid, blocks of 4, worked by hand: block one (0, 4, 1, 5) leaves
    the queue as (8, 2), element 0 having been taken again and skipped; the
    next block grows from the queue's first entry, 8: then 12 (tied with 9 at
    one shared face, queued first), 9, and 13 (two shared faces)."""
    blocks = greedy_partition(grid_neighbours(4), 4)
    assert blocks[0] == [0, 4, 1, 5]
    assert blocks[1] == [8, 12, 9, 13]


def check_greedy_choices(nb, blocks):
    """Every element after a block's first is, at the moment it is placed,
    adjacent to the block and shares a maximal number of faces with it among the
    unplaced elements adjacent to the block -- or no unplaced element is
    adjacent to the block at all (the queue ran dry)."""
    nb = np.asarray(nb)
    K = len(nb)
    placed = np.zeros(K, dtype=bool)

    def nbrs(e):
        return [int(f) for f in nb[e] if f >= 0 and f != e]

    for b in blocks:
        members = set()
        for i, e in enumerate(b):
            if i > 0:
                count = {}
                for m in members:
                    for f in nbrs(m):
                        if not placed[f]:
                            count[f] = count.get(f, 0) + 1
                if count:
                    assert e in count and count[e] == max(count.values()), (b, e, count)
            placed[e] = True
            members.add(e)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("l", [1, 3, 7])
def test_path_blocks_follow_the_greedy_rule(seed, l):
    K = 40
    order = np.random.Generator(np.random.PCG64(seed)).permutation(K) if seed else np.arange(K)
    nb = path_neighbours(order)
    blocks = greedy_partition(nb, l)
    check_partition(blocks, K, l)
    check_greedy_choices(nb, blocks)
    pos = np.empty(K, int)
    pos[order] = np.arange(K)
    p = sorted(pos[blocks[0]])                     # the first block is one segment
    assert all(q - r == 1 for r, q in zip(p, p[1:]))


def test_grid_and_mesh_follow_the_greedy_rule():
    check_greedy_choices(grid_neighbours(6), greedy_partition(grid_neighbours(6), 5))
    verts, tets = kuhn_box_mesh(3, 0.1, 0)
    tets = tets[np.random.Generator(np.random.PCG64(4)).permutation(len(tets))]
    EToE = oracle.build_mesh(verts, tets, 1).EToE
    check_greedy_choices(EToE, greedy_partition(EToE, 20))


def test_in_order_path_gives_consecutive_runs():
    blocks = greedy_partition(path_neighbours(np.arange(23)), 5)
    assert blocks == [list(range(i, min(i + 5, 23))) for i in range(0, 23, 5)]


def test_components_are_not_mixed():
    # two paths of 10 (labels 0..9 and 10..19); blocks of 5 stay inside one path
    nb = -np.ones((20, 4), dtype=np.int64)
    for k in range(20):
        if k % 10 > 0:
            nb[k, 0] = k - 1
        if k % 10 < 9:
            nb[k, 1] = k + 1
    blocks = greedy_partition(nb, 5)
    check_partition(blocks, 20, 5)
    for b in blocks:
        assert len({e // 10 for e in b}) == 1


def _external_fraction(EToE, perm, l):
    K = len(perm)
    inv = np.empty(K, np.int64)
    inv[perm] = np.arange(K)
    nb = inv[EToE[perm]]
    return float(((nb // l) != (np.arange(K)[:, None] // l)).mean())


def test_box_mesh_locality_recovered_after_shuffle():
    verts, tets = kuhn_box_mesh(6, 0.1, 0)
    K = len(tets)
    shuffle = np.random.Generator(np.random.PCG64(7)).permutation(K)
    om = oracle.build_mesh(verts, tets[shuffle], 1)
    native = _external_fraction(oracle.build_mesh(verts, tets, 1).EToE, np.arange(K), 20)
    shuffled = _external_fraction(om.EToE, np.arange(K), 20)
    perm = partition_order(om.EToE, 20)
    assert sorted(perm) == list(range(K))
    ordered = _external_fraction(om.EToE, perm, 20)
    assert shuffled > 0.9 and ordered < native + 0.1, (native, shuffled, ordered)


def test_block_size_one_and_whole_mesh():
    nb = grid_neighbours(5)
    assert len(greedy_partition(nb, 1)) == 25
    blocks = greedy_partition(nb, 25)
    assert len(blocks) == 1 and sorted(blocks[0]) == list(range(25))
    with pytest.raises(ValueError):
        greedy_partition(nb, 0)
