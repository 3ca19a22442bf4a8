"""The seeded input generators (CPU): shapes, determinism and the sizes the
workloads promise.  The generators hold no method arithmetic."""
import numpy as np

from paper_2411_17229_gb300 import synth


def test_zipf_component_weights_match_the_stated_list_sizes():
    w = synth.WORKLOADS["c4_zipf_10m_d768"]
    wts = synth.component_weights(w)
    assert wts.shape == (16384,) and abs(wts.sum() - 1.0) < 1e-12
    ranks = np.sort(wts)[::-1]
    expect = np.arange(1, 16385, dtype=np.float64) ** -1.1
    assert np.allclose(ranks, expect / expect.sum(), rtol=1e-12)
    sizes = wts * w.n
    assert int(sizes.max()) == 1471633 and int(np.median(sizes)) == 72 and int(sizes.min()) == 34


def test_weighted_mixture_is_deterministic_normalised_and_chunk_stable():
    w = synth.Workload("t", 300_000, 32, 10, 1.5, 64, 0.0, 2.0, 1.0, False, True, 64, (4,), 10, (16,), 0.1,
                       comp_zipf=1.1, lists_are_components=True)
    a, qa, la = synth.make(w)
    b, qb, lb = synth.make(w)
    assert np.array_equal(a, b) and np.array_equal(la, lb) and np.array_equal(qa, qb)
    assert np.allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-5)
    # chunk k is drawn from its own generator seeded by (seed, k), and the labels
    # from one stream: a shorter draw is a prefix of a longer one
    c, _, lc = synth.make(w, n=131072)
    assert np.array_equal(lc, la[:131072]) and np.array_equal(c, a[:131072])
    counts = np.bincount(la, minlength=64)
    assert counts.argmax() == int(np.argmax(synth.component_weights(w)))


def test_component_lists_deal_each_component_to_its_own_lists():
    rng = np.random.default_rng(0)
    labels = rng.integers(0, 8, 50_000).astype(np.int32)
    assign = synth.component_lists(labels, 64)
    assert np.array_equal(assign // 8, labels)
    assert np.bincount(assign, minlength=64).min() > 0
    assert np.array_equal(assign, synth.component_lists(labels, 64))
