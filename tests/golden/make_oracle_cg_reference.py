"""Write tests/golden/oracle_plain_cg_<cfg>.json: iterations and wall time of the
FP64 oracle's plain even-odd CG (Section 2's baseline method, no deflation) on
a benchmark workload.  Calls only the oracle and the seeded input generator.

The benchmark's CPU-baseline leg times a bounded sample of oracle CG
iterations and scales it by this iteration count to a time per right-hand side.

usage: python tests/golden/make_oracle_cg_reference.py c2
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle, num_threads  # noqa: E402
from paper_2502_00152_gb300 import inputs as I  # noqa: E402

# the benchmark's source for right-hand side 0 (Gaussian complex source, seed 11)
SOURCE_SEED = 11


def main(name: str) -> None:
    c = I.lattice_config(name)
    dims, m, tol = c["dims"], c["mass"], c["tol"]
    fat, lng = I.hisq_links(dims, c["seed"], c["eps"])
    o = Oracle(dims, fat, lng, t_antiperiodic=True)
    eta = I.gaussian_source(dims, SOURCE_SEED, 0)
    t0 = time.time()
    psi, st = o.solve(m, eta, tol, maxiter=200000)
    wall = time.time() - t0
    out = dict(config=name, dims=list(dims), mass=m, tol=tol, source="gaussian seed 11 source 0",
               t_antiperiodic=True, iterations=st["iterations"], converged=st["converged"],
               full_residual=st["full_residual"], wall_seconds=wall, threads=num_threads())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_plain_cg_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c2")
