"""Writes kl_workload_oracle_qoi.txt: the oracle's QoIs (FP64 Newton with
sparse direct solves) for the scenarios of the KL random-field workload
(4096 scenarios over levels 0..5, KL fields) that the bench compares its
mixed-precision results with.  Calls only oracle/ and the input generator.

    python tests/golden/make_kl_workload_oracle_qoi.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import henry as oh  # noqa: E402
from paper_2302_07804_gb300 import inputs  # noqa: E402

# (level, index) of the picked scenarios: the first and the middle sample of
# levels 0, 1 and 2 of the workload's counts (3264, 656, 128, ...); the
# workload draws level l's inputs as inputs.kl_inputs(KL_TAG0 + l, count).
COUNTS = (3264, 656, 128)
KL_TAG0 = 500
PICKS = ((0, 0), (0, 1632), (1, 0), (1, 328), (2, 0), (2, 64))


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kl_workload_oracle_qoi.txt")
    rows = []
    for level, i in PICKS:
        th = inputs.kl_inputs(KL_TAG0 + level, COUNTS[level])[i]
        q, ok = oh.solve_scenario(oh.Params(), level, th, model="kl")
        assert ok, (level, i)
        rows.append("%d %d %.17e %.17e" % (level, i, q[0], q[1]))
        print(rows[-1], flush=True)
    with open(out, "w") as f:
        f.write("# Oracle QoIs (salt mass [kg/m], c(1.5, 0.25)) of scenarios of the KL workload\n")
        f.write("# (inputs.kl_inputs(500 + level, count)[index]; written by make_kl_workload_oracle_qoi.py)\n")
        f.write("# level index mass c\n")
        f.write("\n".join(rows) + "\n")


if __name__ == "__main__":
    main()
