"""The seeded input generators shared by the oracle tests and the CUDA path:
reproducible from their seeds, with the sizes, ranges and distributions they
state."""
import numpy as np
import pytest
import torch

from paper_2606_08813_b300 import synth


@pytest.mark.parametrize("n,c,dist", [(10_000, 32, "equal"), (1_000_003, 1024, "zipf"), (7, 3, "equal"), (5, 8, "zipf")])
def test_cluster_sizes_largest_remainder(n, c, dist):
    s = synth.cluster_sizes(n, c, dist).numpy()
    assert s.sum() == n and (s >= 0).all()
    p = np.full(c, 1.0 / c) if dist == "equal" else np.arange(1, c + 1, dtype=np.float64) ** -1.1
    p = p / p.sum()
    # largest remainder: every size is the floor or the ceiling of its share
    assert (np.abs(s - p * n) < 1.0).all()
    if dist == "zipf":
        assert (np.diff(s) <= 0).all()


def test_draws_are_pure_functions_of_their_seeds():
    m1 = synth.make_cluster_model(2000, 16, 4, sizes="zipf", seed=3)
    m2 = synth.make_cluster_model(2000, 16, 4, sizes="zipf", seed=3)
    x1, l1 = synth.sample_points(m1, 11)
    x2, l2 = synth.sample_points(m2, 11)
    assert torch.equal(x1, x2) and torch.equal(l1, l2)
    x3, _ = synth.sample_points(m1, 12)
    assert not torch.equal(x1, x3)
    q1, _ = synth.sample_queries(m1, 50, 21)
    q2, _ = synth.sample_queries(m1, 50, 21)
    assert torch.equal(q1, q2)
    assert torch.equal(synth.uniforms(9, 4), synth.uniforms(9, 4))
    assert torch.equal(synth.attributes(100, 5), synth.attributes(100, 5))
    assert torch.equal(synth.range_filters(40, 6), synth.range_filters(40, 6))


def test_points_follow_the_cluster_model():
    m = synth.make_cluster_model(4000, 24, 4, sub_dim=3, decay=0.5, sigma=0.1, seed=7)
    B = m.bases.numpy()
    for c in range(4):
        np.testing.assert_allclose(B[c].T @ B[c], np.eye(3), atol=1e-12)  # orthonormal directions
    X, lab = synth.sample_points(m, 8)
    assert X.dtype == torch.float32 and X.shape == (4000, 24)
    assert np.bincount(lab.numpy(), minlength=4).tolist() == m.sizes.tolist()
    # each cluster's covariance: B diag(decay^(2j)) B^T + sigma^2 I, within sampling error
    for c in range(4):
        Y = X[lab == c].double().numpy()
        cov = np.cov(Y.T)
        want = B[c] @ np.diag([1.0, 0.25, 0.0625]) @ B[c].T + 0.01 * np.eye(24)
        assert np.abs(cov - want).max() < 0.12
        np.testing.assert_allclose(Y.mean(0), m.means[c].numpy(), atol=0.15)


def test_captured_fraction_closed_form():
    # eigenvalues 1 + s2, 0.25 + s2, then s2 (d - 2 times); top 2 over the trace
    d, s2 = 10, 0.01
    want = (1.25 + 2 * s2) / (1.25 + d * s2)
    assert synth.expected_captured_fraction(d, 2, 0.5, 0.1, 2) == pytest.approx(want, rel=1e-12)
    assert synth.expected_captured_fraction(d, 2, 0.5, 0.1, d) == pytest.approx(1.0)


def test_subsets_attributes_and_ranges():
    t = synth.train_subset(1000, 100, 3).numpy()
    assert len(t) == 100 and (np.diff(t) > 0).all() and t.min() >= 0 and t.max() < 1000
    assert synth.train_subset(50, 100, 3).tolist() == list(range(50))
    u = synth.uniforms(1000, 2).numpy()
    assert u.dtype == np.float64 and (u >= 0).all() and (u < 1).all()
    span = 1 << 20
    a = synth.attributes(5000, 1, span=span).numpy()
    assert a.min() >= 0 and a.max() < span
    R = synth.range_filters(2000, 9, span=span, selectivity=0.2, frac_filtered=0.5).numpy()
    i64 = np.iinfo(np.int64)
    full = (R[:, 0] == i64.min) & (R[:, 1] == i64.max)
    part = ~full
    assert 0.4 < part.mean() < 0.6
    width = int(span * 0.2)
    assert (R[part, 1] - R[part, 0] + 1 == width).all()
    assert (R[part, 0] >= 0).all() and (R[part, 1] < span).all()
    # a filtered query keeps about `selectivity` of uniform attributes
    keep = ((a[None] >= R[part][:50, :1]) & (a[None] <= R[part][:50, 1:])).mean()
    assert abs(keep - 0.2) < 0.01
