"""permanova_sW_noalloc: s_W for callers that may not allocate device memory
(plugins of frameworks that own every device allocation, processes confined
to a fixed memory pool).  It runs with the library's fixed resident scratch
array and must give the same s_W as permanova_sW and as the FP64 oracle, call
after call, although every call reuses (and overwrites) the same array; rows
of 1,024 and 2,048 uint8 labels take its perm-block kernel, the others its
brute-force kernel.

This file is collected last so that a failure here cannot hide any other
test's result in a run that stops at the first failure.  It passes alone in a
fresh process (the first call on the device does the array's set-up) and
after the other tests.
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
    torch.cuda.set_device(0)
    c = pm.Context(0)
    yield c
    c.close()


def _case(n, K, P, seed):
    rng = np.random.default_rng(seed)
    D = synth.euclidean_matrix(rng.standard_normal((n, 5)))
    sizes = synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)), min_size=1)
    obs = synth.observed_labels(sizes, seed + 1)
    rows = synth.shuffled_rows(obs, P, seed + 2)
    w = synth.inv_sizes(obs, K)
    return D, rows, w


@pytest.mark.parametrize("n,K,P,seed", [(1001, 4, 37, 1), (257, 3, 300, 2), (130, 7, 5, 4),
                                        (1024, 5, 600, 5), (2048, 3, 100, 6)])
def test_noalloc_matches_permanova_sW_and_oracle_twice(ctx, n, K, P, seed):
    D, rows, w = _case(n, K, P, seed)
    ref_oracle = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    Dd = torch.from_numpy(D).cuda()
    lab = torch.from_numpy(rows.astype(np.uint8)).cuda()
    wd = torch.from_numpy(w).cuda()
    ref = torch.empty(P, dtype=torch.float64, device="cuda")
    pm.permanova_sW(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd, ref)
    pm.permanova_sync(ctx.handle)
    ref = ref.cpu().numpy()
    for _ in range(2):   # two calls in a row share (and reuse) the same scratch
        out = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
        pm.permanova_sW_noalloc(Dd, n, n, lab, pm.LABEL_U8, K, P, wd, out)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=RTOL)
        np.testing.assert_allclose(got, ref_oracle, rtol=RTOL)


@pytest.mark.parametrize("n,K,P,seed", [(1024, 300, 50, 7), (1000, 9, 40, 8)])
def test_noalloc_uint16_labels(ctx, n, K, P, seed):
    """uint16 labels: rows of 1,024 (2,048 bytes) take the perm-block kernel,
    rows of 1,000 (2,000 bytes, not a 16-byte multiple) the brute force;
    both against the FP64 oracle, twice in a row."""
    rng = np.random.default_rng(seed)
    D = synth.euclidean_matrix(rng.standard_normal((n, 5)))
    rows = rng.integers(0, K, size=(P, n)).astype(np.int32)
    w = rng.uniform(0.01, 1.0, K).astype(np.float32)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    Dd = torch.from_numpy(D).cuda()
    lab = torch.from_numpy(rows.astype(np.uint16).view(np.int16)).cuda()
    wd = torch.from_numpy(w).cuda()
    for _ in range(2):
        out = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
        pm.permanova_sW_noalloc(Dd, n, n, lab, pm.LABEL_U16, K, P, wd, out)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL)


def test_noalloc_rejects_oversized_calls(ctx):
    D, rows, w = _case(64, 2, 4, 3)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_sW_noalloc(torch.from_numpy(D).cuda(), 64, 64,
                                torch.from_numpy(rows.astype(np.uint8)).cuda(), pm.LABEL_U8, 2,
                                2_000_000, torch.from_numpy(w).cuda(), out)
    assert ei.value.status == pm.EINVAL
    assert "no-allocation scratch" in str(ei.value)
