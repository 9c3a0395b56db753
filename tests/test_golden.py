"""Frozen oracle outputs (tests/golden/, written by tests/golden/make_golden.py
from the oracle alone): the oracle must keep producing them, and the CUDA path
must match them (labels bit-exact, exact integer sums bit-exact, test
statistics within the stated tolerance)."""
import os
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if not ln.startswith("#")]


def _kv(name):
    return {k: v for k, v in _rows(name)}


def test_oracle_reproduces_golden_permutations():
    obs37 = make_golden.golden_inputs()[0]
    want = np.array(_rows("permutations_n37.txt"), dtype=np.int64)
    got = oracle.permutations(obs37, 20, 9013)
    assert np.array_equal(got, want)


def test_oracle_reproduces_golden_exact_sums():
    _, D16, lab16, rows16, _, _ = make_golden.golden_inputs()
    import synth
    want = np.array([float.fromhex(r[0]) for r in _rows("sW_integer_n16.txt")])
    got = oracle.sW_alg1(D16, rows16, 3, synth.inv_sizes(lab16, 3).astype(np.float64))
    assert np.array_equal(got, want)


def test_oracle_reproduces_golden_test():
    *_, D60, lab60 = make_golden.golden_inputs()
    kv = _kv("test_euclid_n60.txt")
    res = oracle.permanova_test(D60, lab60, 2, 99, 31)
    assert res["s_T"] == float.fromhex(kv["s_T"])
    assert res["s_W"][0] == float.fromhex(kv["s_W_obs"])
    assert res["n_ge"] == int(kv["n_ge"])


@pytest.mark.gpu
def test_cuda_path_matches_golden():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_04556_gb300 as pm
    import synth
    pm.build()
    obs37, D16, lab16, rows16, D60, lab60 = make_golden.golden_inputs()
    with pm.Context(0) as ctx:
        out = torch.empty((21, 37), dtype=torch.int32, device="cuda")
        pm.permanova_permutations(ctx.handle, torch.from_numpy(obs37).cuda(), 37, 4, 20, 9013, out,
                                  pm.LABEL_I32)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), np.array(_rows("permutations_n37.txt"), dtype=np.int32))
        want = np.array([float.fromhex(r[0]) for r in _rows("sW_integer_n16.txt")])
        for form in (pm.FORM_BRUTE, pm.FORM_PERMBLOCK, pm.FORM_GEMM, pm.FORM_AUTO):
            ctx.set_form(form)
            got = ctx.sW(torch.from_numpy(D16).cuda(), torch.from_numpy(rows16).cuda(), 3,
                         torch.from_numpy(synth.inv_sizes(lab16, 3)).cuda())
            pm.permanova_sync(ctx.handle)
            assert np.array_equal(got.cpu().numpy(), want)
        ctx.set_form(pm.FORM_AUTO)
        kv = _kv("test_euclid_n60.txt")
        res = ctx.test(torch.from_numpy(D60).cuda(), torch.from_numpy(lab60).cuda(), 2, 99, 31)
        assert abs(res["s_T"] - float.fromhex(kv["s_T"])) <= 1e-5 * float.fromhex(kv["s_T"])
        assert res["n_ge"] == int(kv["n_ge"])
        assert res["p_value"] == float.fromhex(kv["p_value"])
