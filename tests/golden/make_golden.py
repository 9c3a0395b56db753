"""Write the frozen oracle outputs in tests/golden/.

Calls only ``oracle`` (and ``synth`` for seeded inputs).  The paper prints no
worked example, so these fixtures are the oracle's own results, frozen once
it passed its pins (tests/test_oracle_pins.py), as regression anchors for the
oracle and parity targets for the CUDA path:

* permutations_n37.txt  -- Sec. 1's permutation test: rows 0..20 of the
  Philox4x32-10 Fisher-Yates stream (seed 9013) for a 37-object grouping.
* sW_integer_n16.txt    -- Algorithm 1 (Sec. 2) on an integer matrix with
  power-of-two groups; the sums are exact, stored as hex floats.
* test_euclid_n60.txt   -- the permutation test (s_T, s_W, F, p) on a seeded
  60-object Euclidean case with 99 permutations.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def golden_inputs():
    obs37 = synth.observed_labels([15, 12, 7, 3], 12)
    D16 = synth.integer_matrix(16, 15, 7)
    lab16 = synth.observed_labels([8, 4, 4], 8)
    rows16 = synth.shuffled_rows(lab16, 6, 9)
    X60 = synth.gaussian_points(synth.observed_labels([30, 30], 3), 4, 0.5, 4)
    lab60 = synth.observed_labels([30, 30], 3)
    return obs37, D16, lab16, rows16, synth.euclidean_matrix(X60), lab60


def main():
    obs37, D16, lab16, rows16, D60, lab60 = golden_inputs()
    perms = oracle.permutations(obs37, 20, 9013)
    with open(os.path.join(HERE, "permutations_n37.txt"), "w") as f:
        f.write("# Sec. 1 permutation test (labels reassigned at random): "
                "oracle.permutations(observed, 20, seed=9013); row 0 = observed\n")
        for r in perms:
            f.write(" ".join(str(int(x)) for x in r) + "\n")
    sW = oracle.sW_alg1(D16, rows16, 3, synth.inv_sizes(lab16, 3).astype(np.float64))
    with open(os.path.join(HERE, "sW_integer_n16.txt"), "w") as f:
        f.write("# Sec. 2, Algorithm 1 (s_W): oracle.sW_alg1 on synth.integer_matrix(16, 15, 7), "
                "6 label rows; exact\n")
        for v in sW:
            f.write(float(v).hex() + "\n")
    res = oracle.permanova_test(D60, lab60, 2, 99, 31)
    with open(os.path.join(HERE, "test_euclid_n60.txt"), "w") as f:
        f.write("# Sec. 1 permutation test with Sec. 2's s_W: "
                "oracle.permanova_test(D60, labels, K=2, P=99, seed=31)\n")
        f.write(f"s_T {float(res['s_T']).hex()}\n")
        f.write(f"s_W_obs {float(res['s_W'][0]).hex()}\n")
        f.write(f"F_obs {float(res['F'][0]).hex()}\n")
        f.write(f"n_ge {res['n_ge']}\n")
        f.write(f"p_value {float(res['p_value']).hex()}\n")


if __name__ == "__main__":
    main()
