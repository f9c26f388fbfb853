"""The output blocks the tensor-core products run (pcv_distribution_tc_blocks,
host only), checked on the CPU against brute force: every output of the
requested range is produced by exactly one (row, column) pair of one block
that the kernel keeps, at the canonical index of the merged mode list.

Each side's digit tensor is rebuilt here from the documented orders (table
levels lexicographic, the level n-e entries grouped by seam mode, the
e-photon vectors grouped by their largest mode ascending in side 0's tensor
and by their smallest mode descending in side 1's), so the test also pins the
layout the kernels index.  A pair of a level product is always an output; a
pair of an extension block is one when the column's seam mode lies on the
row's side of the seam (the `cge` comparison), as in the kernel's drain.
"""
import itertools
import math

import pytest

TBM = 128


def msets(w, k):
    return 1 if k == 0 else (0 if w <= 0 else math.comb(w + k - 1, k))


def rank(m, s):
    r, prev, n = 0, 0, len(s)
    for p, x in enumerate(s):
        r += sum(msets(m - v, n - p - 1) for v in range(prev, x))
        prev = x
    return r


def lex(vals, k):
    return [tuple(c) for c in itertools.combinations_with_replacement(vals, k)]


def by_max(vals, k):
    """k-multisets of vals grouped by largest element ascending, lexicographic within."""
    out = []
    for g in vals:
        out += [c + (g,) for c in itertools.combinations_with_replacement([v for v in vals if v <= g], k - 1)]
    return out


def by_min(vals, k, descending):
    out = []
    for g in (reversed(vals) if descending else vals):
        out += [(g,) + c for c in itertools.combinations_with_replacement([v for v in vals if v >= g], k - 1)]
    return out


def tensors(m, n, head):
    h, e, L = head["h"], head["e"], head["L"]
    sides = [list(range(h)), list(range(h, m))]
    ts, seam_lists = [], {}
    for s in (0, 1):
        t = []
        for k in range(e + 1, n - e):
            assert head["lev"][s][k] == len(t), (s, k)
            t += lex(sides[s], k)
        assert head["rows_off"][s] == len(t)
        rows = by_max(sides[0], L) if s == 0 else by_min(sides[1], L, descending=False)
        assert head["nrows"][s] == len(rows)
        seam_lists[s] = [(r, r[-1] if s == 0 else r[0]) for r in rows]
        t += rows
        assert head["cols_off"][s] == len(t)
        vecs = by_max(list(range(m)), e) if s == 0 else by_min(list(range(m)), e, descending=True)
        assert head["ncols"] == len(vecs)
        seam_lists[2 + s] = [(v, v[-1] if s == 0 else v[0]) for v in vecs]
        t += vecs
        assert head["wdig"][s] == len(t)
        ts.append(t)
    return ts, seam_lists


def check(pcv, m, n, lo, hi):
    head, blocks = pcv.abi.pcv_distribution_tc_blocks(m, n, lo, hi)
    ts, seam_lists = tensors(m, n, head)
    N = msets(m, n)
    hi = N if hi < 0 else hi
    seen = {}
    tiles = 0
    assert len(blocks) == head["blocks"] <= 72                 # the kernel's block table
    for b in blocks:
        rt, ct = ts[0 if b["rows_low"] else 1], ts[1 if b["rows_low"] else 0]
        assert b["tile0"] == tiles
        # what the kernel reads stays inside the tensors and the seam lists
        assert b["tn"] in (16, 32, 48, 64)
        assert 0 <= b["rows0"] < b["rows"] and 0 <= b["cols0"] < b["cols"]
        assert 0 <= b["row_off"] and b["row_off"] + b["rows"] <= len(rt)
        assert 0 <= b["col_off"] and b["col_off"] + b["cols"] <= len(ct)
        if b["kind"] == 1:
            assert 0 <= b["ri_off"] and b["ri_off"] + b["rows"] <= len(seam_lists[b["rs"]])
            assert 0 <= b["ci_off"] and b["ci_off"] + b["cols"] <= len(seam_lists[b["cs"]])
        tiles += -(-(b["rows"] - b["rows0"]) // TBM) * -(-(b["cols"] - b["cols0"]) // b["tn"])
        for r in range(b["rows0"], b["rows"]):
            R = rt[b["row_off"] + r]
            for c in range(b["cols0"], b["cols"]):
                C = ct[b["col_off"] + c]
                if b["kind"] == 1:
                    rm, rkey = seam_lists[b["rs"]][b["ri_off"] + r]
                    cm, ckey = seam_lists[b["cs"]][b["ci_off"] + c]
                    assert rm == R and cm == C           # the seam index names the same entry
                    if (ckey < rkey) if b["cge"] else (ckey > rkey):
                        continue
                o = rank(m, tuple(sorted(R + C)))
                if lo <= o < hi:
                    seen[o] = seen.get(o, 0) + 1
    assert tiles == head["tiles"]
    assert sorted(seen) == list(range(lo, hi)), (m, n, lo, hi)
    assert set(seen.values()) <= {1}, [o for o, c in seen.items() if c > 1][:5]
    return head


@pytest.fixture(scope="module")
def pcv():
    import paper_2204_00602_gb300 as pcv
    return pcv


@pytest.mark.parametrize("m,n", [(2, 2), (3, 2), (2, 3), (5, 4), (6, 3), (7, 4), (9, 5), (8, 6), (12, 6),
                                 (10, 7), (7, 8), (6, 9), (5, 10), (20, 3)])
def test_every_output_once_whole(pcv, m, n):
    check(pcv, m, n, 0, -1)


@pytest.mark.parametrize("m,n", [(7, 4), (9, 5), (12, 6), (8, 8)])
def test_every_output_once_in_parts(pcv, m, n):
    N = msets(m, n)
    cuts = sorted({0, 1, N // 7, N // 3, N // 2, N - 2, N})
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        check(pcv, m, n, lo, hi)


def test_bench_workload_layout(pcv):
    """m=20, n=10: e = 3, the digit tensors hold levels 4..6, the 11,440 level-7
    entries and the 1,540 three-photon vectors per side; the plan's tiles
    cover the 20,030,010 outputs with at most 14 % padding."""
    head, blocks = pcv.abi.pcv_distribution_tc_blocks(20, 10)
    assert (head["e"], head["L"], head["h"]) == (3, 7, 10)
    assert head["nrows"] == [11440, 11440] and head["ncols"] == 1540
    assert head["wdig"] == [715 + 2002 + 5005 + 11440 + 1540] * 2
    assert [head["lev"][0][k] for k in range(4, 7)] == [0, 715, 715 + 2002]
    useful = math.comb(29, 10) / (TBM * 64)
    assert useful <= head["tiles"] <= 1.14 * useful


def test_range_split_tile_counts_at_bench_size(pcv):
    """m=20, n=10 split into P equal ranges: the level blocks keep close to
    their share, the extension blocks run 1.6x / 2.7x / 5.0x the whole call's
    tiles in total at P = 2 / 4 / 8 (the high side's e-photon vectors are in
    max-grouped order, so a range's lexicographic run of them is scattered)."""
    N = math.comb(29, 10)

    def tiles(blocks, kind):
        return sum(-(-(b["rows"] - b["rows0"]) // TBM) * -(-(b["cols"] - b["cols0"]) // b["tn"])
                   for b in blocks if b["kind"] == kind)

    _, whole = pcv.abi.pcv_distribution_tc_blocks(20, 10)
    for P, lev_max, ext_ratio in ((2, 1.01, 1.60), (4, 1.09, 2.74), (8, 1.16, 5.02)):
        parts = [pcv.abi.pcv_distribution_tc_blocks(20, 10, N * r // P, N * (r + 1) // P)[1] for r in range(P)]
        assert sum(tiles(b, 0) for b in parts) <= lev_max * tiles(whole, 0)
        assert sum(tiles(b, 1) for b in parts) == pytest.approx(ext_ratio * tiles(whole, 1), rel=0.01)


def test_every_output_once_in_seeded_random_ranges(pcv):
    """Seeded random sizes (n = 2 .. 10, at most 30,000 outputs) and random
    ranges, including empty and one-output ranges."""
    import random
    rng = random.Random(2204)
    cases = 0
    while cases < 12:
        n = rng.randint(2, 10)
        m = rng.randint(2, 14)
        N = msets(m, n)
        if N > 30_000:
            continue
        a, b = sorted(rng.randrange(N + 1) for _ in range(2))
        for lo, hi in ((a, b), (a, a), (a, min(N, a + 1))):
            check(pcv, m, n, lo, hi)
        cases += 1
