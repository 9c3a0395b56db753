"""permanova_sW_noalloc: s_W for callers that cannot allocate device memory
(graph capture without allocation nodes, frameworks that own every device
allocation, fixed memory pools).  It runs with the library's fixed resident
scratch array and must give the same s_W as permanova_sW, call after call.

This file is collected last so that a failure here cannot hide any other
test's result in a run that stops at the first failure.
"""
import numpy as np
import pytest

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
    return (torch.from_numpy(D).cuda(), torch.from_numpy(rows.astype(np.uint8)).cuda(),
            torch.from_numpy(synth.inv_sizes(obs, K)).cuda())


def test_noalloc_matches_permanova_sW_twice(ctx):
    for n, K, P, seed in ((1001, 4, 37, 1), (257, 3, 300, 2)):
        D, lab, w = _case(n, K, P, seed)
        ref = torch.empty(P, dtype=torch.float64, device="cuda")
        pm.permanova_sW(ctx.handle, D, n, n, lab, pm.LABEL_U8, K, P, w, ref)
        pm.permanova_sync(ctx.handle)
        for _ in range(2):   # two calls in a row share (and reuse) the same scratch
            out = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
            pm.permanova_sW_noalloc(D, n, n, lab, pm.LABEL_U8, K, P, w, out)
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=RTOL)


def test_noalloc_rejects_oversized_calls(ctx):
    D, lab, w = _case(64, 2, 4, 3)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_sW_noalloc(D, 64, 64, lab, pm.LABEL_U8, 2, 2_000_000, w, out)
    assert ei.value.status == pm.EINVAL
    assert "no-allocation scratch" in str(ei.value)
