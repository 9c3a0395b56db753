"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (default kernel plan, uint8 label rows, the benchmark's batch sizes).

* n = 1,000 / 999 rows and n = 20,000 / 3,999 rows: sampled rows against the
  FP64 oracle (Algorithm 1) one by one.
* n = 50,000 Bray-Curtis / 8,192 rows: 64 rows spread over the launch (both
  ends, every label-row tile position in between) against the oracle.
* n = 25,145 Jaccard / 4,000 rows (the paper's own workload shape, Sec. 3):
  64 sampled rows against the oracle.
* n = 100,000 / 8,192 rows (the headline workload): 512 rows spread over
  the launch against Huygens' identity for Euclidean distances, s_W =
  sum_g sum_{i in g} |x_i - mu_g|^2 computed from the generating points in
  FP64 (a property that holds at any size).
* the whole permutation test at n = 100,000 with 99,999 permutations in one
  call: 256 rows against Huygens' identity, s_T against its closed form, the
  count and p against the returned s_W values.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2505_04556_gb300 as pm  # noqa: E402

RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


def _run(ctx, cfg, X, n_rows, seed):
    D = synth.recipe_matrix_device(cfg, X)
    lab = synth.device_label_rows(cfg["labels"], n_rows, seed, dtype=torch.uint8)
    w = torch.from_numpy(cfg["w"]).cuda()
    out = torch.empty(n_rows, dtype=torch.float64, device="cuda")
    pm.permanova_sW(ctx.handle, D, cfg["n"], cfg["n"], lab, pm.LABEL_U8, cfg["K"], n_rows, w, out)
    pm.permanova_sync(ctx.handle)
    return D, lab, out.cpu().numpy()


def _oracle_rows(D, lab, cfg, idx):
    Dh = D.cpu().numpy()
    rows = lab[idx].cpu().numpy().astype(np.int32)
    return oracle.sW_alg1(Dh, rows, cfg["K"], cfg["w"].astype(np.float64))


@pytest.mark.parametrize("name,n_rows,sample", [("euclid-1k", 999, 999), ("euclid-20k", 3999, 48)])
def test_full_size_sampled_rows(ctx, name, n_rows, sample):
    cfg = synth.recipe(name)
    X = synth.recipe_points(cfg)
    D, lab, got = _run(ctx, cfg, X, n_rows, 31)
    idx = np.unique(np.linspace(0, n_rows - 1, sample).astype(int))
    ref = _oracle_rows(D, lab, cfg, idx)
    np.testing.assert_allclose(got[idx], ref, rtol=RTOL)


def _spread(n_rows, count):
    """``count`` label rows spread over a launch: both ends, the first and last
    rows of several label-row tiles, and evenly spaced rows in between."""
    idx = {0, 1, 24, 25, 127, 128, n_rows - 2, n_rows - 1}
    idx.update(int(round(k * (n_rows - 1) / (count - 1))) for k in range(count))
    k = 3
    while len(idx) < count:           # fill up with odd offsets if rounding collided
        idx.add((k * 7919) % n_rows)
        k += 1
    return np.array(sorted(idx))


def test_full_size_braycurtis_50k(ctx):
    cfg = synth.recipe("braycurtis-50k")
    X = synth.recipe_points(cfg)
    D, lab, got = _run(ctx, cfg, X, 8192, 32)
    idx = _spread(8192, 64)
    assert len(idx) >= 64
    ref = _oracle_rows(D, lab, cfg, idx)
    np.testing.assert_allclose(got[idx], ref, rtol=RTOL)


def test_full_size_jaccard_25k(ctx):
    cfg = synth.recipe("jaccard-25k")
    X = synth.recipe_points(cfg)
    D, lab, got = _run(ctx, cfg, X, 4000, 34)
    idx = _spread(4000, 64)
    assert len(idx) >= 64
    ref = _oracle_rows(D, lab, cfg, idx)
    np.testing.assert_allclose(got[idx], ref, rtol=RTOL)


def test_full_size_euclid_100k_huygens(ctx):
    cfg = synth.recipe("euclid-100k")
    X = synth.recipe_points(cfg)
    D, lab, got = _run(ctx, cfg, X, 8192, 33)
    K, dim = cfg["K"], X.shape[1]
    # Huygens: s_W = sum_g (sum_{i in g} |x_i|^2 - |sum_{i in g} x_i|^2 / n_g)
    sq = np.einsum("ij,ij->i", X, X)
    for r in np.linspace(0, 8191, 512).astype(int):
        g = lab[r].cpu().numpy().astype(np.int64)
        cnt = np.bincount(g, minlength=K).astype(np.float64)
        sums = np.stack([np.bincount(g, weights=X[:, d], minlength=K) for d in range(dim)], axis=1)
        closed = float(np.sum(np.bincount(g, weights=sq, minlength=K)) -
                       np.sum(np.einsum("kd,kd->k", sums, sums) / cnt))
        assert abs(got[r] - closed) <= RTOL * closed, (r, got[r], closed)


def test_full_size_permanova_test_100k(ctx):
    """The whole permutation test at the headline size in one permanova_test
    call: n = 100,000, K = 10, 99,999 permutations (device permutations, the
    s_W pass over all 100,000 label rows, s_T, F, the count).  s_W of 256 rows
    spread over the 100,000 against Huygens' identity from the generating
    points (the rows regenerated with permanova_permutations from the same
    seed), s_T against its one-group closed form sum_i |x_i - mu|^2, and the
    count and p against the returned s_W values."""
    cfg = synth.recipe("euclid-100k")
    X = synth.recipe_points(cfg)
    D = synth.recipe_matrix_device(cfg, X)
    n, K, P, seed = cfg["n"], cfg["K"], cfg["P"], 4321
    obs = torch.from_numpy(np.ascontiguousarray(cfg["labels"], dtype=np.int32)).cuda()
    out = torch.empty(P + 1, dtype=torch.float64, device="cuda")
    res = pm.permanova_test(ctx.handle, D, n, n, obs, K, P, seed, out)
    sW = out.cpu().numpy()
    n_ge = int(np.sum(sW[1:] <= sW[0]))
    assert res["n_perms"] == P
    assert res["n_ge"] == n_ge and res["p_value"] == (1 + n_ge) / (1 + P)
    mu = X.mean(axis=0)
    s_T = float(np.sum((X - mu) ** 2))
    assert abs(res["s_T"] - s_T) <= RTOL * s_T
    del D
    torch.cuda.empty_cache()
    lab = torch.empty((P + 1, n), dtype=torch.uint8, device="cuda")
    pm.permanova_permutations(ctx.handle, obs, n, K, P, seed, lab, pm.LABEL_U8)
    torch.cuda.synchronize()
    sq = np.einsum("ij,ij->i", X, X)
    dim = X.shape[1]
    for r in np.linspace(0, P, 256).astype(int):
        g = lab[r].cpu().numpy().astype(np.int64)
        cnt = np.bincount(g, minlength=K).astype(np.float64)
        sums = np.stack([np.bincount(g, weights=X[:, d], minlength=K) for d in range(dim)], axis=1)
        closed = float(np.sum(np.bincount(g, weights=sq, minlength=K)) -
                       np.sum(np.einsum("kd,kd->k", sums, sums) / cnt))
        assert abs(sW[r] - closed) <= RTOL * closed, (r, sW[r], closed)
