"""The seeded input generators (CPU): every workload recipe has the sizes the
benchmark and the parity tests assume, the distance generators agree with
SciPy's definitions of the same distances, the device builders (run here on
torch's CPU backend) give the host builders' matrices, and every label row is
a permutation of the observed grouping.  These inputs feed both the oracle and
the CUDA path, so a mistake here would go unseen by the parity tests."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

WORKLOADS = {   # name: (n, K, P)
    "euclid-1k": (1000, 3, 999),
    "euclid-20k": (20000, 4, 3999),
    "braycurtis-50k": (50000, 8, 9999),
    "jaccard-25k": (25145, 5, 3999),
    "euclid-100k": (100000, 10, 99999),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_recipe_sizes(name):
    n, K, P = WORKLOADS[name]
    cfg = synth.recipe(name)
    assert (cfg["n"], cfg["K"], cfg["P"]) == (n, K, P)
    sizes = np.asarray(cfg["sizes"])
    assert sizes.shape == (K,) and sizes.sum() == n and sizes.min() >= 1
    lab = cfg["labels"]
    assert lab.shape == (n,) and lab.dtype == np.int32
    assert np.array_equal(np.bincount(lab, minlength=K), sizes)
    np.testing.assert_allclose(cfg["w"], (1.0 / sizes).astype(np.float32), rtol=0)
    # the same seed gives the same workload
    assert np.array_equal(synth.recipe(name)["labels"], lab)


def test_largest_remainder_sizes():
    for n, props, m in [(10, [1, 1, 1], 1), (1000, [40, 30, 20, 10], 1), (25145, [35, 25, 20, 12, 8], 1),
                        (17, [0.9, 0.05, 0.05], 3)]:
        s = synth.largest_remainder_sizes(n, props, min_size=m)
        assert s.sum() == n and s.min() >= m
        p = np.asarray(props, float) / np.sum(props)
        quota = m + p * (n - m * len(props))
        assert np.all(np.abs(s - quota) < 1.0)
    with pytest.raises(ValueError):
        synth.largest_remainder_sizes(5, [1, 1, 1], min_size=2)


def test_distance_generators_match_scipy():
    dist = pytest.importorskip("scipy.spatial.distance")
    lab = synth.observed_labels([40, 35, 25], 3)
    X = synth.gaussian_points(lab, 8, 0.3, 1)
    np.testing.assert_allclose(synth.euclidean_matrix(X), dist.squareform(dist.pdist(X, "euclidean")),
                               rtol=2e-7, atol=2e-6)
    C = synth.dirichlet_compositions(lab, features=50, seed=2)
    np.testing.assert_allclose(synth.braycurtis_matrix(C), dist.squareform(dist.pdist(C, "braycurtis")),
                               rtol=2e-7, atol=1e-7)
    B = synth.presence_features(lab, features=120, seed=3)
    J = synth.jaccard_matrix(B)
    np.testing.assert_allclose(J, dist.squareform(dist.pdist(B, "jaccard")), rtol=2e-7, atol=1e-7)
    assert J.min() >= 0.0 and J.max() <= 1.0


@pytest.mark.parametrize("name", ["euclid-1k", "braycurtis-50k", "jaccard-25k"])
def test_device_builder_matches_host_builder(name):
    """recipe_matrix_device (the builder of the full-size matrices) against
    recipe_matrix_host on a scaled copy of the workload, on torch's CPU
    backend: the same matrix up to the rounding of the last fp32 bit."""
    cfg = synth.recipe(name, n=300, P=4)
    X = synth.recipe_points(cfg)
    H = synth.recipe_matrix_host(cfg, X)
    D = synth.recipe_matrix_device(cfg, X, device="cpu", chunk=64).numpy()
    assert D.shape == H.shape == (300, 300) and D.dtype == np.float32
    np.testing.assert_allclose(D, H, rtol=1e-6, atol=1e-6)
    assert np.all(np.diag(D) == 0) and np.allclose(D, D.T, rtol=1e-6, atol=1e-6)


def test_label_rows_are_permutations():
    obs = synth.observed_labels([7, 5, 3, 1], 11)
    rows = synth.shuffled_rows(obs, 50, 4)
    assert rows.shape == (50, 16) and rows.dtype == np.int32
    assert np.array_equal(rows[0], obs)
    assert np.all(np.sort(rows, axis=1) == np.sort(obs))
    assert len({r.tobytes() for r in rows}) > 40          # distinct orders
    assert np.array_equal(synth.shuffled_rows(obs, 50, 4), rows)
    dev = synth.device_label_rows(obs, 50, 4, device="cpu", dtype=torch.int32, chunk=7).numpy()
    assert np.array_equal(dev[0], obs)
    assert np.all(np.sort(dev, axis=1) == np.sort(obs))


def test_integer_and_poisoned_matrices():
    D = synth.integer_matrix(40, 15, 5)
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)
    assert np.all(D == np.round(D)) and D.min() >= 0 and D.max() <= 15
    E = synth.poison_lower(D)
    iu = np.triu_indices(40, 1)
    assert np.array_equal(E[iu], D[iu]) and np.all(np.isnan(E[np.tril_indices(40)]))
