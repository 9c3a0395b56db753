"""Failure detection without a GPU fault: a device wait that nothing completes
runs out after a short limit, the kernel returns, the host reads ETIMEOUT,
and the context keeps working.  Invalid input is reported as an error code,
never as a trap."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2505_04556_gb300 as pm  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


def test_bounded_wait_times_out_and_context_survives(ctx):
    pm.permanova_selftest_wait(ctx.handle, 200_000)        # 0.2 s limit
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_sync(ctx.handle)
    assert ei.value.status == pm.ETIMEOUT
    pm.permanova_sync(ctx.handle)                            # error word was cleared
    rng = np.random.default_rng(2)
    D = synth.euclidean_matrix(rng.standard_normal((300, 4)))
    obs = synth.observed_labels([150, 100, 50], 3)
    rows = synth.shuffled_rows(obs, 40, 4)
    w = synth.inv_sizes(obs, 3)
    for form in (pm.FORM_BRUTE, pm.FORM_PERMBLOCK, pm.FORM_GEMM):
        ctx.set_form(form)
        out = ctx.sW(torch.from_numpy(D).cuda(), torch.from_numpy(rows.astype(np.uint8)).cuda(), 3,
                     torch.from_numpy(w).cuda())
        pm.permanova_sync(ctx.handle)
        np.testing.assert_allclose(out.cpu().numpy(), oracle.sW_alg1(D, rows, 3, w.astype(np.float64)),
                                   rtol=1e-5)
    ctx.set_form(pm.FORM_AUTO)


def test_selftest_limit_validated(ctx):
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_selftest_wait(ctx.handle, 0)
    assert ei.value.status == pm.EINVAL
