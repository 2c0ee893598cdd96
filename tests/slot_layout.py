"""The library's particle slot layout, restated for the tests from its ABI
description (include/polypic.h, polypic_num_keys and polypic_sort).

This is NOT the oracle.  The oracle sorts particles by the plain cell index
(k n_y + j) n_x + i and fixes, per cell, the list of its particles in
increasing index order (a stable sort).  The library additionally arranges
cells and particles in a layout of its own (an implementation device the paper
does not have), and the GPU tests check that layout here as a format property:

  * keys order cells in tiles of 8 x 8 x 4 cells (row-major tile order); a
    tile is 2 x 2 x 2 blocks of 4 x 4 x 2 cells (x fastest); cells inside a
    block are x fastest:  key = tile * 256 + block_in_tile * 32 + cell_in_block;
  * slots follow the stable (key, index) order, except that inside every
    block of 32 consecutive keys round r = 0, 1, ... lists the r-th particle of
    every key of the block holding more than r particles, keys ascending.

Everything here is vectorised NumPy so that it also runs at full size.
"""
import numpy as np

import oracle


def tiles(n):
    return ((int(n[0]) + 7) // 8, (int(n[1]) + 7) // 8, (int(n[2]) + 3) // 4)


def num_keys(n) -> int:
    t = tiles(n)
    return t[0] * t[1] * t[2] * 256


def tile_key(i, j, k, n):
    """Key of cell (i, j, k) (scalars or integer arrays)."""
    i, j, k = (np.asarray(v, dtype=np.int64) for v in (i, j, k))
    tx, ty, _ = tiles(n)
    tile = ((k // 4) * ty + (j // 8)) * tx + (i // 8)
    blk = ((i // 4) % 2) + 2 * ((j // 4) % 2) + 4 * ((k // 2) % 2)
    cell = (i % 4) + 4 * (j % 4) + 16 * (k % 2)
    return tile * 256 + blk * 32 + cell


def key_of_cell_index(c, n):
    """Library key of the oracle's plain cell index c = (k n_y + j) n_x + i."""
    c = np.asarray(c, dtype=np.int64)
    nx, ny = int(n[0]), int(n[1])
    return tile_key(c % nx, (c // nx) % ny, c // (nx * ny), n)


def library_order(x32, n, dx):
    """(perm, cell_start, key) of the library's documented slot layout, built
    from the oracle's stable per-cell particle lists: perm[j] = particle in
    slot j, cell_start over the library's keys, key[p] = library key of p."""
    perm, cs, cidx = oracle.cell_sort(x32, n, dx)
    P = perm.shape[0]
    key = key_of_cell_index(cidx, n)
    # rank of each particle inside its cell's stable list
    rank = np.empty(P, dtype=np.int64)
    rank[perm.astype(np.int64)] = np.arange(P, dtype=np.int64) - cs[cidx[perm]].astype(np.int64)
    # blocks of 32 keys ascending; inside a block round by round, keys ascending
    order = np.lexsort((key, rank, key // 32))
    nk = num_keys(n)
    counts = np.bincount(key, minlength=nk)
    cstart = np.zeros(nk + 1, dtype=np.int64)
    np.cumsum(counts, out=cstart[1:])
    return (order.astype(np.uint32), cstart.astype(np.uint32), key.astype(np.uint32))


def per_cell_lists_match(gpu_perm, x32, n, dx) -> bool:
    """The GPU's slot order, read cell by cell (the oracle decides each
    particle's cell), lists every cell's particles exactly as the oracle's
    stable sort does: the part of the order that the method fixes."""
    perm, _, cidx = oracle.cell_sort(x32, n, dx)
    gp = np.asarray(gpu_perm, dtype=np.int64)
    if gp.shape[0] != perm.shape[0]:
        return False
    if gp.shape[0] == 0:
        return True
    if not np.array_equal(np.sort(gp), np.arange(gp.shape[0])):
        return False
    grouped = gp[np.argsort(cidx[gp], kind="stable")]
    return bool(np.array_equal(grouped, perm.astype(np.int64)))
