"""Writes the regression fixtures of this directory from the CPU oracle alone (oracle/ and
the seeded data generator; nothing from the CUDA path).  Run from the repository root:

    python tests/golden/make_golden.py

The paper prints no worked numeric example (its decoding example is a figure), so these
values are the oracle's own results on fixed seeded inputs: they guard the oracle against
unintended change and give the GPU tests fixed targets.  A change to them must come with a
change of the oracle's arithmetic justified by a passage of the paper."""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2311_06952_gb300 import datagen  # noqa: E402


def deoct_workload0():
    """Algorithm 4 (DEOCT) on the tiny workload: depth 2, P = 64, G = 100, M = 0.5, CR = 0.9,
    Philox seed 0, stream 0."""
    w = datagen.make_workload(0)
    ranks, nu = oracle.encode(w["X"])
    r = oracle.de_run(ranks, nu, w["y"], w["K"], depth=w["depth"], P=w["P"], G=w["G"], M=w["M"],
                      CR=w["CR"], seed=w["seed"], history=True)
    best = r["best"]
    a, th = oracle.decode(r["pop"][best:best + 1], w["depth"], nu)
    return {
        "cite": "Algorithm 4 (DEOCT), Eqs. mutation / crossover / selection, Eq. aenc, Eq. benc",
        "inputs": "datagen.make_workload(0): n=1000, F=8, K=2; depth 2, P=64, G=100, M=0.5, CR=0.9, seed 0",
        "best_index": int(best),
        "best_fitness_per_generation": [float(x) for x in r["best_fit_hist"]],
        "best_tree_a": [int(x) for x in a[0]],
        "best_tree_theta": [int(x) for x in th[0]],
        "final_population_sha256": hashlib.sha256(r["pop"].tobytes()).hexdigest(),
        "final_fitness_sha256": hashlib.sha256(r["fit"].tobytes()).hexdigest(),
    }


def eval_workload1():
    """Algorithm 1 class counts of the population-evaluation workload at full size."""
    w = datagen.make_workload(1)
    ranks, nu = oracle.encode(w["X"])
    a, th = datagen.random_population(nu, w["P"], w["depth"],
                                      np.random.Generator(np.random.PCG64(w["pop_seed"])))
    counts = oracle.eval_counts(ranks, w["y"], w["K"], a, th, w["depth"])
    _, err, _, _ = oracle.fitness(counts, a, w["X"].shape[0])
    return {
        "cite": "Algorithm 1 (class counts Zhat) and the loss identity of Section 2",
        "inputs": "datagen.make_workload(1): n=1e5, F=20, K=3; 256 random depth-3 trees, pop_seed 7",
        "counts_sha256": hashlib.sha256(np.ascontiguousarray(counts, np.uint32).tobytes()).hexdigest(),
        "errors": [int(x) for x in err],
    }


def main():
    for name, fn in (("deoct_workload0.json", deoct_workload0), ("eval_workload1.json", eval_workload1)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")
        print("wrote", name)


if __name__ == "__main__":
    main()
