"""Host model of the cluster kernel's grid bound (no GPU).

The cluster-pair kernel launches one one-warp block per possible super-cluster: the grid is
N / (8 NC) + nrows + 1 blocks (NC = 8 clusters of 8 particles per super-cluster in the FP32
forms, 4 in the FP64 form; integer division), and blocks past the last super-cluster only
write zero energy partials. A row of n particles holds ceil(n / 8) clusters and
ceil(ceil(n / 8) / NC) super-clusters, so the bound must hold for every way of spreading N
particles over the rows, including the adversarial ones: every row one particle past a full
super-cluster, or one particle per row.
"""
import numpy as np


def supers(counts, nc):
    clusters = -(-counts // 8)
    return int((-(-clusters // nc)).sum())


def bound(N, nrows, nc):
    return N // (8 * nc) + nrows + 1


def test_grid_bound_covers_every_row_occupancy():
    rng = np.random.default_rng(7)
    for nc in (8, 4):
        for _ in range(2000):
            nrows = int(rng.integers(1, 4000))
            kind = rng.integers(0, 4)
            if kind == 0:    # uniform
                counts = rng.poisson(rng.uniform(0.1, 600), nrows)
            elif kind == 1:  # one past a full super-cluster in every row
                counts = 8 * nc * rng.integers(0, 5, nrows) + 1
            elif kind == 2:  # one particle per row, some empty
                counts = (rng.random(nrows) < 0.9).astype(np.int64)
            else:            # one dense row, the rest sparse
                counts = rng.integers(0, 3, nrows)
                counts[rng.integers(0, nrows)] += int(rng.integers(0, 200000))
            counts = counts.astype(np.int64)
            N = int(counts.sum())
            assert supers(counts, nc) <= bound(N, nrows, nc), (nc, nrows, N)


def test_bound_is_tight_for_one_past_full():
    """Rows of 8 NC k + 1 particles need the bound's per-row term: its slack is then only the
    extra particles' own share, nrows // (8 NC), plus the final 1."""
    for nc in (8, 4):
        nrows, k = 1000, 3
        counts = np.full(nrows, 8 * nc * k + 1, np.int64)
        N = int(counts.sum())
        assert supers(counts, nc) == nrows * (k + 1)
        assert bound(N, nrows, nc) - supers(counts, nc) == nrows // (8 * nc) + 1
