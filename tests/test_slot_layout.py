"""Host-only checks of the tests' restatement of the library's slot layout
(tests/slot_layout.py), so that the GPU sort tests compare against what the
ABI header describes: keys are a bijection on cells, every 4x4x2 block and
every 8x8x4 tile occupies one contiguous key range in row-major tile order,
and inside a block the slots deal each cell's stable particle list round by
round."""
import itertools

import numpy as np

import oracle
import slot_layout


def test_keys_are_a_bijection_with_contiguous_blocks_and_tiles():
    n = (16, 16, 8)
    nk = slot_layout.num_keys(n)
    keys = {}
    for i, j, k in itertools.product(range(n[0]), range(n[1]), range(n[2])):
        keys[(i, j, k)] = int(slot_layout.tile_key(i, j, k, n))
    assert len(set(keys.values())) == len(keys) == nk
    for bi, bj, bk in itertools.product(range(4), range(4), range(4)):
        ks = sorted(keys[(4 * bi + a, 4 * bj + b, 2 * bk + c)]
                    for a in range(4) for b in range(4) for c in range(2))
        assert ks == list(range(ks[0], ks[0] + 32)) and ks[0] % 32 == 0
        # x fastest inside the block
        assert keys[(4 * bi + 1, 4 * bj, 2 * bk)] == ks[0] + 1
        assert keys[(4 * bi, 4 * bj + 1, 2 * bk)] == ks[0] + 4
        assert keys[(4 * bi, 4 * bj, 2 * bk + 1)] == ks[0] + 16
    for ti, tj, tk in itertools.product(range(2), range(2), range(2)):
        ks = sorted(keys[(8 * ti + a, 8 * tj + b, 4 * tk + c)]
                    for a in range(8) for b in range(8) for c in range(4))
        assert ks[0] == 256 * ((tk * 2 + tj) * 2 + ti)
        assert ks == list(range(ks[0], ks[0] + 256))


def test_ragged_grid_keys_stay_below_num_keys():
    n = (20, 12, 10)
    ii, jj, kk = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    keys = slot_layout.tile_key(ii.ravel(), jj.ravel(), kk.ravel(), n)
    assert len(np.unique(keys)) == keys.size
    assert keys.max() < slot_layout.num_keys(n)
    c = (kk * n[1] + jj) * n[0] + ii
    assert np.array_equal(slot_layout.key_of_cell_index(c.ravel(), n), keys)


def test_library_order_deals_the_stable_cell_lists_round_by_round():
    rng = np.random.default_rng(90)
    n = (16, 8, 8)
    dx = 1 / 16
    x = np.stack([rng.uniform(1, n[b] - 1, 3000) * dx for b in range(3)]).astype(np.float32)
    x[:, :400] = np.array([[5.5], [3.5], [2.5]]) * dx      # one crowded cell
    perm_cells, cs_cells, cidx = oracle.cell_sort(x, n, dx)
    out, cs, key = slot_layout.library_order(x, n, dx)
    nk = slot_layout.num_keys(n)
    assert np.array_equal(np.sort(out), np.arange(x.shape[1]))
    assert slot_layout.per_cell_lists_match(out, x, n, dx)
    assert np.array_equal(np.diff(cs.astype(np.int64)), np.bincount(key, minlength=nk))
    for b in range(nk // 32):
        lo, hi = cs[32 * b], cs[32 * b + 32]
        seg = out[lo:hi]
        assert np.all(key[seg] // 32 == b)
        kk = key[seg]
        rank = np.zeros_like(kk)
        for k in np.unique(kk):
            rank[kk == k] = np.arange(np.sum(kk == k))
            c = int(cidx[seg[kk == k][0]])
            assert np.array_equal(seg[kk == k], perm_cells[cs_cells[c]:cs_cells[c + 1]])
        # round r holds every key's r-th particle, keys ascending
        assert np.array_equal(np.lexsort((kk, rank)), np.arange(len(seg)))


def test_per_cell_check_rejects_a_swap_inside_a_cell():
    rng = np.random.default_rng(5)
    n = (8, 8, 8)
    dx = 1 / 8
    x = np.stack([rng.uniform(1, 7, 900) * dx for b in range(3)]).astype(np.float32)
    out, _, key = slot_layout.library_order(x, n, dx)
    assert slot_layout.per_cell_lists_match(out, x, n, dx)
    # swap two particles of one cell: the per-cell order is no longer stable
    k = np.bincount(key).argmax()
    slots = np.flatnonzero(key[out] == k)
    bad = out.copy()
    bad[slots[0]], bad[slots[1]] = bad[slots[1]], bad[slots[0]]
    assert not slot_layout.per_cell_lists_match(bad, x, n, dx)
