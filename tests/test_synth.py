"""Input generators: published SplitMix64 outputs, determinism and shapes."""
import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 started from state 0 (Vigna's reference
    # splitmix64.c): 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    assert synth.splitmix_at(0, 0) == 0xE220A8397B1DCDAF
    assert synth.splitmix_at(0, 1) == 0x6E789E6AA1B965F4
    assert synth.splitmix_at(0, 2) == 0x06C45D188009454F


def test_generators_are_deterministic_and_in_range():
    a = synth.rmat_pairs(10, 5000, 7)
    b = synth.rmat_pairs(10, 5000, 7)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert a[0].max() < 1024 and a[1].max() < 1024
    w = synth.weights(10000, 3, 1, 100)
    assert w.min() >= 1 and w.max() <= 100
    assert len(np.unique(w)) == 100
    p = synth.permutation(1000, 9)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_rmat_quadrant_skew():
    s, d = synth.rmat_pairs(16, 200000, 11)
    # top bit of (src, dst) follows the first-level quadrant probabilities
    top_s = (s >> 15) & 1
    top_d = (d >> 15) & 1
    q = np.bincount(top_s * 2 + top_d, minlength=4) / len(s)
    assert np.allclose(q, [0.57, 0.19, 0.19, 0.05], atol=0.01)


def test_dedup_keeps_first_occurrence():
    s = np.array([1, 2, 1, 3, 3, 2], np.uint32)
    d = np.array([2, 2, 2, 3, 1, 2], np.uint32)
    ks, kd = synth.dedup_pairs(s, d, 8, drop_self=False)
    assert ks.tolist() == [1, 2, 3, 3] and kd.tolist() == [2, 2, 3, 1]
    ks, kd = synth.dedup_pairs(s, d, 8, drop_self=True)
    assert ks.tolist() == [1, 3] and kd.tolist() == [2, 1]


def test_grid_edge_count():
    s, d = synth.grid_pairs(4, 5)
    assert len(s) == 2 * (4 * 4 + 5 * 3)
    diff = np.abs(s.astype(int) - d.astype(int))
    assert set(diff.tolist()) == {1, 5}


def test_tiny_workload_shape():
    w = synth.tiny_workload()
    assert len(w.g_src) == 8192 and len(w.ins_src) == 1024
    assert len(w.del_src) == 1024 and len(w.q_src) == 4096
    assert w.g_w.min() >= 1 and w.g_w.max() <= 100
