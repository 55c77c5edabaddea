"""Greedy breadth-first element partition (oracle, integer only).

Test infrastructure only (see the package docstring).

Section 5.2 ("Flux Extraction"), Algorithm 2 (Simple Greedy Partition): the
elements are cut into blocks of at most l elements, each grown from a seed by
repeatedly taking, from a queue of candidates, the element that shares the most
faces with the block being built; the neighbours of every element taken join
the queue.  When a block is full the first entry of the queue seeds the next
block; when the queue runs dry an arbitrary remaining element is added to it.
Numbering the elements block by block puts face neighbours next to each other,
which is what a flux-gather tile needs.

Readings where the algorithm leaves a choice open:
  * ties between candidates sharing the same number of faces go to the one
    that entered the queue first;
  * "a seed element" for the first block and "an arbitrary element" for a dry
    queue are the lowest-numbered element not yet placed;
  * the queue is a set (an element already queued is not queued twice) kept in
    insertion order; an element already placed may be queued again and is
    skipped when it is taken, as in the algorithm.
"""
from __future__ import annotations

import numpy as np


def greedy_partition(nbrs, block: int):
    """Blocks of the greedy partition.

    nbrs: (K, 4) integer array, the neighbour across each face (the element
    itself or a negative number on boundary faces).  Returns a list of blocks
    (lists of element indices) in the order they were built.
    """
    nbrs = np.asarray(nbrs)
    K = nbrs.shape[0]
    if block < 1:
        raise ValueError("block size must be positive")
    placed = np.zeros(K, dtype=bool)
    remaining = K
    lowest = 0
    blocks = []
    carry = None

    def lowest_unplaced():
        nonlocal lowest
        while lowest < K and placed[lowest]:
            lowest += 1
        return lowest

    def face_neighbours(e):
        return [int(f) for f in nbrs[e] if f >= 0 and f != e]

    while remaining:
        seed = carry if carry is not None else lowest_unplaced()
        carry = None
        queue = [seed]
        queued = {seed}
        shared = {}          # faces each element shares with the current block
        current = []
        while True:
            best = 0
            for i in range(1, len(queue)):
                if shared.get(queue[i], 0) > shared.get(queue[best], 0):
                    best = i
            e = queue.pop(best)
            queued.discard(e)
            if not placed[e]:
                placed[e] = True
                remaining -= 1
                current.append(e)
                for f in face_neighbours(e):
                    shared[f] = shared.get(f, 0) + 1
                if len(current) == block:
                    carry = queue[0] if queue else None
                    break
                for f in face_neighbours(e):
                    if f not in queued:
                        queue.append(f)
                        queued.add(f)
            if not queue:
                if remaining == 0:
                    break
                x = lowest_unplaced()
                queue.append(x)
                queued.add(x)
        blocks.append(current)
    return blocks


def partition_order(nbrs, block: int) -> np.ndarray:
    """perm with perm[i] = the element placed at position i (blocks in order)."""
    blocks = greedy_partition(nbrs, block)
    return np.array([e for b in blocks for e in b], dtype=np.int64)
