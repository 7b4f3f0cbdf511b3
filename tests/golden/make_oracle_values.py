"""Write the oracle's values for the full colour-transfer workload.

    python tests/golden/make_oracle_values.py

Calls only the CPU oracle (oracle/) on the seeded synthetic colour-transfer
pair (65,536 points per side, d=3, squared Euclidean, seed 0) in both
decision precisions and stores the NNS work (sum of m_t * n_t), the round
count and R in colour_transfer_oracle.json.  The benchmark reads the work
count to scale its bounded CPU-oracle sample to one full pair.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_07378_gb300 import workloads  # noqa: E402


def main():
    p = workloads.color_transfer(seed=0)
    out = {"generator": "workloads.color_transfer(seed=0, n=65536, clusters=8, sigma=0.08)", "metric": "sql2"}
    for decide in ("fp32", "fp64"):
        t0 = time.perf_counter()
        r = oracle.solve_pair(p, "sql2", decide)
        out[decide] = {"cost": r.cost, "rounds": r.rounds, "pair_evals": r.pair_evals, "nnz": int(r.plan_f.size),
                       "near_ties": r.near_ties, "violations": r.violations, "seconds": time.perf_counter() - t0}
    out["pair_evals"] = out["fp32"]["pair_evals"]
    out["rel_err_fp32_decisions_vs_fp64"] = abs(out["fp32"]["cost"] - out["fp64"]["cost"]) / out["fp64"]["cost"]
    with open(os.path.join(HERE, "colour_transfer_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
