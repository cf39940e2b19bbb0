"""Host logic of the host-buffer batch codec: how chunks are grouped."""
import random

from paper_1503_00638_gb300.hostio import chunk_groups


def test_chunk_groups_cover_in_order_and_respect_the_size():
    rng = random.Random(3)
    for _ in range(200):
        sizes = [rng.randint(1, 1000) for _ in range(rng.randint(0, 40))]
        cap = rng.randint(1, 3000)
        g = chunk_groups(sizes, cap)
        # consecutive, non-empty, covering every chunk once
        if not sizes:
            assert g == []
            continue
        assert [a for a, _ in g] == [0] + [b for _, b in g[:-1]]
        assert g[-1][1] == len(sizes)
        assert all(b > a for a, b in g)
        for a, b in g:
            # within the size unless one chunk alone exceeds it
            assert sum(sizes[a:b]) <= cap or b == a + 1
            # maximal: the next chunk would not have fit
            if b < len(sizes):
                assert sum(sizes[a:b + 1]) > cap


def test_chunk_groups_edge_cases():
    assert chunk_groups([], 10) == []
    assert chunk_groups([50], 10) == [(0, 1)]
    assert chunk_groups([5, 5, 5], 10) == [(0, 2), (2, 3)]
    assert chunk_groups([5, 5, 5], 15) == [(0, 3)]
