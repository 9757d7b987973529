"""A CPU model of how the one-launch loop of small all-pairs pairs spreads its
work over a thread-block cluster (no GPU).

Each iteration of that loop computes the all-pairs kernel's (template block,
source split) items and the epilogue's blocks of points on the cluster's
CTAs: CTA `rank` of `ncta`, sub-block `sub` of 256 / BS, takes items
rank * SUB + sub, + ncta * SUB, ...; the epilogue's virtual blocks go to CTAs
rank, rank + ncta, .... The plan (tile BS x QPT, S source splits of `chunk`
sources) is the all-pairs kernel's own. This model replays those loops and
checks that, for every cluster size, every item runs exactly once, every
(template point, source) pair is summed exactly once (the source tiles read
past N fall in the zero-mass padding of the staged copy) and every template
point gets exactly one epilogue, so the loop computes what the separate
launches compute.
"""
import itertools

import numpy as np
import pytest

SMS = 152
NT = 256  # threads per CTA, the epilogue's block size


def plan_direct(N, M, bs, qpt):
    qblocks = -(-M // (bs * qpt))
    target = 4 * SMS
    S = max(1, -(-target // qblocks))
    tiles = -(-N // bs)
    S = min(S, max(tiles, 1), 64)
    tiles_per = -(-tiles // S)
    chunk = tiles_per * bs
    S = max(1, -(-N // chunk))
    return qblocks, S, chunk


def epilogue_blocks(M):
    return max(1, min(-(-M // NT), 2 * SMS))


def cluster_size(items, sub, nblk, max_cl=16):
    return min(max(-(-items // sub), nblk, 1), max_cl)


CASES = [(1000, 1000), (1500, 555), (4096, 256), (64, 16384), (50, 1), (1, 37), (129, 130), (3000, 300)]
TILES = [(128, 1), (128, 2), (128, 4), (256, 1), (256, 2), (256, 4)]


@pytest.mark.parametrize("N,M", CASES)
@pytest.mark.parametrize("bs,qpt", TILES)
def test_items_points_and_sources_are_covered_once(N, M, bs, qpt):
    assert N <= 4096 and M <= 16384 and N * M <= 1 << 20
    qblocks, S, chunk = plan_direct(N, M, bs, qpt)
    items = qblocks * S
    sub_n = NT // bs
    nblk = epilogue_blocks(M)
    npad = -(-N // bs) * bs
    for ncta in sorted({1, 2, 5, 8, cluster_size(items, sub_n, nblk)}):
        seen = np.zeros(items, dtype=int)
        pair_count = np.zeros((M, N), dtype=np.int16)
        for rank, sub in itertools.product(range(ncta), range(sub_n)):
            for w in range(rank * sub_n + sub, items, ncta * sub_n):
                seen[w] += 1
                qb, split = w % qblocks, w // qblocks
                j0 = split * chunk
                j1 = min(N, j0 + chunk)
                for b in range(j0, j1, bs):
                    assert b + bs <= npad  # the tile stays in the staged copy
                    src = np.arange(b, min(b + bs, N))
                    for t, q in itertools.product(range(bs), range(qpt)):
                        i = qb * bs * qpt + t + q * bs
                        if i < M:
                            pair_count[i, src] += 1
        assert np.all(seen == 1)
        assert np.all(pair_count == 1)
        epi = np.zeros(M, dtype=int)
        for rank in range(ncta):
            for b in range(rank, nblk, ncta):
                for tid in range(NT):
                    epi[np.arange(b * NT + tid, M, nblk * NT)] += 1
        assert np.all(epi == 1)


def test_staged_sources_fit_in_shared_memory():
    # the packed layout takes 32 bytes per source, padded to a whole tile
    for bs in (128, 256):
        npad = -(-4096 // bs) * bs
        assert npad * 32 + 8 * 1024 <= 227 * 1024
