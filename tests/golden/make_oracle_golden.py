"""Writes tests/golden/tiny_two_source_oracle.json: the FP64 oracle's total ELBO, local
objectives and gradients on the two-source 5 x 48 x 48 case (seed 2026), so that any
later change of the oracle's arithmetic shows up as a failing regression test and has
to be justified.  Calls only oracle/ and the input generator.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle  # noqa: E402
from paper_1801_10277_gb300 import synth  # noqa: E402


def main():
    prob = synth.config(0)
    orc = Oracle(prob)
    tot, loc = orc.elbo(prob.theta)
    _, g, _ = orc.derivs(prob.theta)
    out = {"workload": prob.name, "seed": 2026, "elbo_total": tot, "elbo_local": loc.tolist(),
           "grad": g.tolist(),
           "note": "FP64 oracle values (log x! dropped); regression fixture, not a paper value"}
    with open(os.path.join(HERE, "tiny_two_source_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
