"""Pins for the oracle's post-acquisition reorder (Sec. 2): a hand-written
example, the transpose written with numpy axes, and the round trip."""
import numpy as np

from paper_1503_00638_gb300 import synth


def test_hand_example(orc):
    # 2 time samples of 3 series: rows (t) -> columns
    a = np.array([[1, 2, 3], [4, 5, 6]], dtype=np.int32)
    assert orc.reorder_time(a).tolist() == [[1, 4], [2, 5], [3, 6]]


def test_against_numpy_axes_and_round_trip(orc):
    rng = np.random.default_rng(1)
    for dt in (np.uint8, np.uint16, np.float32, np.complex64):
        a = rng.integers(0, 200, size=(7, 5, 3)).astype(dt)
        r = orc.reorder_time(a)
        assert r.shape == (5, 3, 7)
        assert np.array_equal(r, np.moveaxis(a, 0, -1))
        # back: view the output as [S][T] -> [T][S]
        back = orc.reorder_time(r.reshape(15, 7)).reshape(7, 5, 3)
        assert np.array_equal(back, a)


def test_reorder_then_round_equals_rounding_the_time_fastest_cube(orc):
    cfg = synth.VisConfig(3, 5, 16, 2 ** 12, 0.05, seed=2)
    v = synth.visibilities(cfg)                 # [F][P][T]
    tslow = np.ascontiguousarray(np.moveaxis(v, -1, 0))   # [T][F][P]
    assert np.array_equal(orc.reorder_time(tslow), v)
    r1 = orc.reduce_precision(orc.reorder_time(tslow), cfg.n_samp, cfg.f)
    r2 = orc.reduce_precision_c64(v, cfg.n_samp, cfg.f)
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))
