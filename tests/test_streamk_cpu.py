"""Arithmetic of the stream-K split that the RPY pair kernel's tile sums rely on
(no GPU): W work units (tile, source chunk) are split over G CTAs, CTA b owning
units [floor(bW/G), floor((b+1)W/G)); the CTA that completes a tile reads the
partials of the tile's CTAs, which it finds as the range [owner(u0), owner(u1)]
of the owners of the tile's first and last unit (G <= W), or as the owners of
the tile's units one by one (G > W, where a CTA owns at most one unit and some
own none), with owner(u) = ceil((u + 1) G / W) - 1. Checked here against the
partition itself, by brute force over small W and G and a ragged tile list."""
import numpy as np


def unit_start(b, W, G):
    return (b * W) // G


def owner(u, W, G):
    return -(-((u + 1) * G) // W) - 1


def test_owner_is_the_cta_whose_range_holds_the_unit():
    for W in range(1, 80):
        for G in range(1, 120):
            starts = [unit_start(b, W, G) for b in range(G + 1)]
            for u in range(W):
                b = owner(u, W, G)
                assert 0 <= b < G
                assert starts[b] <= u < starts[b + 1], (W, G, u, b)


def test_tile_partials_are_found_in_both_regimes():
    rng = np.random.default_rng(3)
    for _ in range(200):
        chunks = rng.integers(1, 9, size=rng.integers(1, 12))   # units per tile (ragged)
        off = np.concatenate([[0], np.cumsum(chunks)])
        W = int(off[-1])
        for G in sorted({1, 2, W // 3 + 1, W, W + 1, 2 * W + 5, 7 * W}):
            starts = [unit_start(b, W, G) for b in range(G + 1)]
            for t in range(len(chunks)):
                u0, u1 = int(off[t]), int(off[t + 1]) - 1
                # the CTAs that wrote a partial of tile t: those owning one of its units
                truth = sorted({b for b in range(G) if starts[b] < starts[b + 1]
                                and starts[b] <= u1 and starts[b + 1] > u0})
                if G > W:
                    assert all(starts[b + 1] - starts[b] <= 1 for b in range(G))
                    found = [owner(u, W, G) for u in range(u0, u1 + 1)]
                else:
                    assert all(starts[b + 1] > starts[b] for b in range(G))
                    found = list(range(owner(u0, W, G), owner(u1, W, G) + 1))
                assert found == truth, (W, G, t)
                # the units each CTA adds to the tile's counter sum to the tile's units
                covered = sum(min(starts[b + 1], u1 + 1) - max(starts[b], u0) for b in truth)
                assert covered == u1 - u0 + 1
