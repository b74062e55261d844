"""Candidate features (host code of the library, no GPU needed)."""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W


@pytest.fixture(scope="module")
def rc():
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


def items_of(rc, seed):
    pk = W.proposal_kernel(seed)
    bc = rc.compile(pk.src)
    return [(bc, G, S, pk.instance(G, S, i).globals) for (G, S, i) in W.proposal_candidates(seed)]


def test_shape_range_and_thread_invariance(rc):
    items = items_of(rc, 5)
    a = rc.features(items, n_threads=1)
    b = rc.features(items, n_threads=7)
    assert a.shape == (64, 128) and a.dtype == np.float32
    np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(a)) and a.min() >= 0.0
    # launch-shape block follows the candidate: log2 S / 10, log2 G / 6, S / 1024, G / 64
    for f, (_, G, S, _) in zip(a, items):
        assert f[109] == pytest.approx(np.log2(S) / 10, abs=1e-6)
        assert f[110] == pytest.approx(np.log2(G) / 6, abs=1e-6)
        assert f[112] == pytest.approx(S / 1024, abs=1e-6) and f[113] == pytest.approx(G / 64, abs=1e-6)


def test_opcode_histogram_sums_to_one(rc):
    items = items_of(rc, 2)
    f = rc.features(items[:4])
    np.testing.assert_allclose(f[:, :52].sum(axis=1), 1.0, rtol=1e-5)
    assert np.all(f[:, :52] == f[0, :52])  # a property of the kernel, not the candidate


def test_sampled_collisions_track_the_oracle(rc, oracle):
    """Where every work-item is evaluated (N <= 4096), the sampled-race
    feature agrees with the oracle's verdict on nearly every candidate."""
    agree = total = 0
    for s in range(12):
        pk = W.proposal_kernel(s)
        items = items_of(rc, s)
        f = rc.features(items)
        for k, (_, G, S, g) in enumerate(items):
            if G * S > 2048:
                continue
            r = oracle.check(pk.src, G, S, g)
            agree += int((r["status"] == 1) == (f[k, 107] > 0))
            total += 1
    assert total > 100 and agree / total >= 0.95, (agree, total)


def test_rejects_bad_inputs(rc):
    pk = W.proposal_kernel(0)
    bc = rc.compile(pk.src)
    with pytest.raises(rc.RaceCheckError):
        rc.features([(bc, 1, 32, [np.zeros(4, np.int32)])])  # two globals declared, one given
    with pytest.raises(rc.RaceCheckError):
        rc.features([(bc, 1, 2048, pk.instance(1, 32, 0).globals)])
