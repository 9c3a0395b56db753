"""Seeded synthetic inputs for PERMANOVA workloads.

This module only makes inputs: points, distance matrices, group sizes and label
rows.  It holds none of the method's arithmetic (no within-group sums, no
test statistics) and is the one module that both the oracle-side tests and the
CUDA-side tests/benchmark draw inputs from.

The shapes follow the paper's statement of typical workloads (Sec. 2: distance
matrices between 1k^2 and 100k^2 elements, 1k to 1M permutations) and its own
benchmark (Sec. 3: a dense fp32 matrix of 25,145 objects, 3,999 permutations),
whose UniFrac data is not available; the generators below stand in for it:

* Gaussian points in R^d, group g shifted by +shift along axis (g mod d),
  Euclidean distances (configurations of n = 1,000 / 20,000 / 100,000).
* Dirichlet(0.5) compositions of 200 features, group g boosting the alpha of
  its own 10-feature block by 1.5x, Bray-Curtis distances (n = 50,000).
* integer-valued symmetric matrices with small entries, for exact sums.

Label rows for ``permanova_sW`` are uniformly random permutations of an
observed grouping drawn with numpy's PCG64 (input generation only; the
permutation test's own Philox stream lives in the library and the oracle).
"""
from __future__ import annotations

import numpy as np

SEED_POINTS = 1234
SEED_ORDER = 5678
SEED_PERMS = 9012


def largest_remainder_sizes(n: int, props, min_size: int = 1) -> np.ndarray:
    """Integer group sizes summing to n, proportional to ``props`` (Hamilton's
    largest-remainder rounding), each at least ``min_size``."""
    props = np.asarray(props, dtype=np.float64)
    props = props / props.sum()
    K = len(props)
    if n < K * min_size:
        raise ValueError("n too small for the requested minimum group size")
    base = min_size * np.ones(K, dtype=np.int64)
    rest = n - base.sum()
    quota = props * rest
    fl = np.floor(quota).astype(np.int64)
    rem = rest - fl.sum()
    order = np.argsort(-(quota - fl), kind="stable")
    fl[order[:rem]] += 1
    return base + fl


def dirichlet_sizes(n: int, K: int, alpha: float, seed: int, min_size: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return largest_remainder_sizes(n, rng.dirichlet(alpha * np.ones(K)), min_size)


def observed_labels(sizes, seed: int) -> np.ndarray:
    """Labels 0..K-1 with the given group sizes, object order shuffled."""
    sizes = np.asarray(sizes, dtype=np.int64)
    lab = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    rng = np.random.default_rng(seed)
    rng.shuffle(lab)
    return lab


def gaussian_points(labels, dim: int, shift: float, seed: int) -> np.ndarray:
    """x_i ~ N(0, I_dim) + shift * e_{(label_i mod dim)}; float64."""
    labels = np.asarray(labels)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((labels.shape[0], dim))
    X[np.arange(labels.shape[0]), labels % dim] += shift
    return X


def euclidean_matrix(X) -> np.ndarray:
    """Dense fp32 Euclidean distance matrix (zero diagonal), computed in float64."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    sq = np.einsum("ij,ij->i", X, X)
    D = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, 2048):
        r1 = min(n, r0 + 2048)
        D2 = sq[r0:r1, None] + sq[None, :] - 2.0 * (X[r0:r1] @ X.T)
        np.maximum(D2, 0.0, out=D2)
        D[r0:r1] = np.sqrt(D2)
    np.fill_diagonal(D, 0.0)
    return D


def dirichlet_compositions(labels, features: int = 200, alpha: float = 0.5,
                           boost: float = 1.5, block: int = 10, seed: int = 0) -> np.ndarray:
    """Rows ~ Dirichlet(alpha * 1), with group g's alpha on features
    [block*g, block*g + block) (mod features) multiplied by ``boost``."""
    labels = np.asarray(labels)
    rng = np.random.default_rng(seed)
    n = labels.shape[0]
    A = np.full((n, features), alpha, dtype=np.float64)
    cols = (block * labels[:, None] + np.arange(block)[None, :]) % features
    A[np.arange(n)[:, None], cols] *= boost
    G = rng.standard_gamma(A)
    G /= G.sum(axis=1, keepdims=True)
    return G


def braycurtis_matrix(C) -> np.ndarray:
    """Bray-Curtis dissimilarity sum|u-v| / sum(u+v) as fp32 (host, small n)."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    tot = C.sum(axis=1)
    D = np.zeros((n, n), dtype=np.float32)
    for i in range(n):
        D[i] = (np.abs(C[i][None, :] - C).sum(axis=1) / (tot[i] + tot)).astype(np.float32)
    np.fill_diagonal(D, 0.0)
    return D


def presence_features(labels, features: int = 1000, rate: float = 0.3, boost: float = 1.5,
                      block: int = 50, seed: int = 0) -> np.ndarray:
    """Sparse presence/absence profiles (a stand-in for microbiome feature
    tables): feature f present with probability ``rate``, multiplied by
    ``boost`` on the ``block`` features of the object's own group."""
    labels = np.asarray(labels)
    rng = np.random.default_rng(seed)
    n = labels.shape[0]
    p = np.full((n, features), rate)
    cols = (block * labels[:, None] + np.arange(block)[None, :]) % features
    p[np.arange(n)[:, None], cols] = min(1.0, rate * boost)
    return rng.random((n, features)) < p


def jaccard_matrix(B) -> np.ndarray:
    """Jaccard distance 1 - |a & b| / |a | b| between presence rows, fp32 in
    [0, 1] (0 for two empty rows); host, small n."""
    B = np.asarray(B, dtype=np.float64)
    inter = B @ B.T
    cnt = B.sum(axis=1)
    union = cnt[:, None] + cnt[None, :] - inter
    with np.errstate(invalid="ignore", divide="ignore"):
        D = np.where(union > 0, 1.0 - inter / union, 0.0)
    D = D.astype(np.float32)
    np.fill_diagonal(D, 0.0)
    return D


def integer_matrix(n: int, high: int, seed: int) -> np.ndarray:
    """Symmetric fp32 matrix with integer entries in [0, high], zero diagonal."""
    rng = np.random.default_rng(seed)
    U = rng.integers(0, high + 1, size=(n, n)).astype(np.float32)
    D = np.triu(U, 1)
    D = D + D.T
    return D.astype(np.float32)


def poison_lower(D: np.ndarray) -> np.ndarray:
    """Copy of D with the diagonal and the lower triangle set to NaN (never read)."""
    E = np.array(D, dtype=np.float32, copy=True)
    E[np.tril_indices(E.shape[0])] = np.nan
    return E


def shuffled_rows(observed, n_rows: int, seed: int, include_observed: bool = True) -> np.ndarray:
    """``n_rows`` x n int32 label rows, each a uniformly random permutation of
    ``observed`` (row 0 = ``observed`` when ``include_observed``)."""
    obs = np.asarray(observed, dtype=np.int32)
    rng = np.random.default_rng(seed)
    out = np.empty((n_rows, obs.shape[0]), dtype=np.int32)
    start = 0
    if include_observed and n_rows > 0:
        out[0] = obs
        start = 1
    for r in range(start, n_rows):
        out[r] = obs[rng.permutation(obs.shape[0])]
    return out


def inv_sizes(labels, K: int) -> np.ndarray:
    """1/n_g as float32 (0 for an empty group), the paper's inv_group_sizes."""
    cnt = np.bincount(np.asarray(labels).ravel(), minlength=K)[:K].astype(np.float64)
    w = np.zeros(K, dtype=np.float64)
    nz = cnt > 0
    w[nz] = 1.0 / cnt[nz]
    return w.astype(np.float32)


# ---------------------------------------------------------------------------
# Workload recipes.  Each returns a dict with the observed labels, group
# sizes, K, P and a way to build D.  ``n`` may be overridden to make a scaled
# copy of a workload for fast tests.
# ---------------------------------------------------------------------------

def recipe(name: str, n: int | None = None, P: int | None = None) -> dict:
    if name == "euclid-1k":          # n=1,000, R^16, K=3 sizes 400/350/250, P=999
        n = n or 1000
        sizes = largest_remainder_sizes(n, [400, 350, 250])
        cfg = dict(dim=16, kind="euclid", K=3, P=P or 999, label_type="i32", idx=1)
    elif name == "euclid-20k":       # n=20,000, R^32, K=4 at 40/30/20/10 %, P=3,999
        n = n or 20000
        sizes = largest_remainder_sizes(n, [40, 30, 20, 10])
        cfg = dict(dim=32, kind="euclid", K=4, P=P or 3999, label_type="u8", idx=2)
    elif name == "braycurtis-50k":   # n=50,000 Dirichlet(0.5) x 200, K=8, P=9,999
        n = n or 50000
        sizes = largest_remainder_sizes(n, [25, 20, 15, 12, 10, 8, 6, 4])
        cfg = dict(dim=200, kind="braycurtis", K=8, P=P or 9999, label_type="u8", idx=3)
    elif name == "jaccard-25k":      # the paper's benchmark shape: n=25,145, P=3,999
        n = n or 25145               # distances in [0, 1] from sparse presence profiles
        sizes = largest_remainder_sizes(n, [35, 25, 20, 12, 8])
        cfg = dict(dim=1000, kind="jaccard", K=5, P=P or 3999, label_type="u8", idx=5)
    elif name == "euclid-100k":      # n=100,000, R^16, K=10 Dirichlet(2) sizes, P=99,999
        n = n or 100000
        sizes = dirichlet_sizes(n, 10, 2.0, SEED_POINTS + 4, min_size=2)
        cfg = dict(dim=16, kind="euclid", K=10, P=P or 99999, label_type="u8", idx=4)
    else:
        raise KeyError(name)
    idx = cfg["idx"]
    labels = observed_labels(sizes, SEED_ORDER + idx)
    cfg.update(name=name, n=n, sizes=sizes, labels=labels,
               w=inv_sizes(labels, cfg["K"]), seed_points=SEED_POINTS + idx,
               seed_perms=SEED_PERMS + idx)
    return cfg


def recipe_points(cfg: dict) -> np.ndarray:
    if cfg["kind"] == "euclid":
        return gaussian_points(cfg["labels"], cfg["dim"], 0.3, cfg["seed_points"])
    if cfg["kind"] == "jaccard":
        return presence_features(cfg["labels"], features=cfg["dim"], seed=cfg["seed_points"])
    return dirichlet_compositions(cfg["labels"], features=cfg["dim"], seed=cfg["seed_points"])


def recipe_matrix_host(cfg: dict, X=None) -> np.ndarray:
    X = recipe_points(cfg) if X is None else X
    if cfg["kind"] == "euclid":
        return euclidean_matrix(X)
    if cfg["kind"] == "jaccard":
        return jaccard_matrix(X)
    return braycurtis_matrix(X)


def recipe_matrix_device(cfg: dict, X=None, device="cuda", chunk: int = 4096):
    """The same matrix built on the GPU with torch in float64 (input generation
    for sizes that do not fit a host build; plain torch ops, not the method)."""
    import torch
    X = recipe_points(cfg) if X is None else X
    n = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(device=device, dtype=torch.float64)
    D = torch.empty((n, n), dtype=torch.float32, device=device)
    if cfg["kind"] == "euclid":
        sq = (Xd * Xd).sum(dim=1)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            blk = sq[r0:r1, None] + sq[None, :] - 2.0 * (Xd[r0:r1] @ Xd.T)
            D[r0:r1] = blk.clamp_min_(0.0).sqrt_().to(torch.float32)
    elif cfg["kind"] == "jaccard":
        cnt = Xd.sum(dim=1)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            inter = Xd[r0:r1] @ Xd.T
            union = cnt[r0:r1, None] + cnt[None, :] - inter
            blk = torch.where(union > 0, 1.0 - inter / union.clamp_min(1.0), torch.zeros_like(union))
            D[r0:r1] = blk.to(torch.float32)
    else:
        tot = Xd.sum(dim=1)
        c = max(1, chunk // 16)
        for r0 in range(0, n, c):
            r1 = min(n, r0 + c)
            num = torch.cdist(Xd[r0:r1], Xd, p=1.0)
            D[r0:r1] = (num / (tot[r0:r1, None] + tot[None, :])).to(torch.float32)
    D.fill_diagonal_(0.0)
    return D


def device_label_rows(observed, n_rows: int, seed: int, device="cuda", dtype=None,
                      include_observed: bool = True, chunk: int = 2048):
    """``n_rows`` x n label rows on the GPU, each a random permutation of
    ``observed`` (torch's seeded generator; input generation only)."""
    import torch
    dtype = dtype or torch.uint8
    obs = torch.as_tensor(np.asarray(observed), device=device).to(torch.int64)
    n = obs.shape[0]
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty((n_rows, n), dtype=dtype, device=device)
    start = 0
    if include_observed and n_rows > 0:
        out[0] = obs.to(dtype)
        start = 1
    for r0 in range(start, n_rows, chunk):
        r1 = min(n_rows, r0 + chunk)
        keys = torch.rand((r1 - r0, n), generator=gen, device=device)
        idx = torch.argsort(keys, dim=1)
        out[r0:r1] = obs[idx].to(dtype)
        del keys, idx
    return out
