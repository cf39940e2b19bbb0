"""The device-arena offset allocator (bsgpu_arena_*) is host code: checked on
the CPU against a model of the reserved ranges."""
import random

import pytest

bs = pytest.importorskip("paper_1503_00638_gb300.bsgpu")


def test_basic_alignment_capacity_and_errors():
    a = bs.Arena(10_000, 256)
    assert a.capacity == 9984
    o1 = a.alloc(1)
    o2 = a.alloc(300)
    assert o1 % 256 == 0 and o2 % 256 == 0 and {o1, o2} == {0, 256}
    assert a.stats()["used"] == 256 + 512
    assert a.alloc(10_000) is None            # larger than what is free
    with pytest.raises(bs.BsgpuError):
        a.free(12345)                          # not a range start
    a.free(o1)
    with pytest.raises(bs.BsgpuError):
        a.free(o1)                             # twice
    a.free(o2)
    st = a.stats()
    assert st["used"] == 0 and st["free_ranges"] == 1 and st["largest_free"] == 9984
    assert st["high_water"] == 768
    assert bs._lib.bsgpu_arena_create(1000, 3) is None   # align not a power of two


def test_best_fit_and_coalescing():
    a = bs.Arena(1 << 20, 256)
    offs = [a.alloc(4096) for _ in range(8)]
    for o in offs[1::2]:
        a.free(o)                              # four 4 KiB holes
    small = a.alloc(2048)
    assert small == offs[1]                    # the first smallest hole that fits
    for o in offs[0::2]:
        a.free(o)
    a.free(small)
    st = a.stats()
    assert st["free_ranges"] == 1 and st["largest_free"] == 1 << 20


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_against_model(seed):
    rng = random.Random(seed)
    cap, align = 1 << 24, 512
    a = bs.Arena(cap, align)
    live = {}
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 200):
            off = rng.choice(list(live))
            a.free(off)
            del live[off]
        else:
            n = int(2 ** rng.uniform(0, 20))
            off = a.alloc(n)
            size = -(-max(n, 1) // align) * align
            if off is None:
                # refused only when no free range is large enough
                assert a.stats()["largest_free"] < size
                continue
            assert off % align == 0 and off + size <= cap
            for o, s in live.items():
                assert off + size <= o or o + s <= off, "overlap"
            live[off] = size
        assert a.stats()["used"] == sum(live.values())
    for off in list(live):
        a.free(off)
    st = a.stats()
    assert st["used"] == 0 and st["free_ranges"] == 1 and st["largest_free"] == cap
