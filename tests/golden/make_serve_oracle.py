"""Write tests/golden/serve_pool_oracle.json: the CPU oracle's results on the
served pool (gen.serve_spec, the seed of the served workload), one record per
problem: a digest of the generated inputs and a digest of the oracle's
matching with its pass and cycle counts.

Calls only the oracle and the seeded generators.  The benchmark's served
section compares its outputs with these records (after checking that the
inputs it generated have the recorded digest), so that the large pool is
checked against the oracle without running the oracle at benchmark time.

    python tests/golden/make_serve_oracle.py [pool_size]
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "serve_pool_oracle.json")


def input_digest(g) -> str:
    h = hashlib.sha256()
    for a in (g.colptr, g.rowidx, g.weight, g.mate):
        h.update(memoryview(a).cast("B"))
    return h.hexdigest()[:32]


def mate_digest(mate) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(mate, dtype=np.int32).tobytes()).hexdigest()[:32]


def _one(spec):
    sys.path[:0] = [ROOT]
    import oracle
    from paper_1801_09809_gb300 import gen
    g = gen.build_spec(spec)
    out, st, _ = oracle.get().improve(g)
    return {"spec": list(spec), "n": g.n, "nnz": g.nnz, "input": input_digest(g),
            "mate": mate_digest(out), "iterations": st["iterations"],
            "cycles_applied": st["cycles_applied"]}


def main(pool_size: int = 128):
    sys.path[:0] = [ROOT]
    import oracle
    from paper_1801_09809_gb300 import gen
    oracle.build()
    specs = gen.serve_spec(pool_size, seed=gen.SEED_BASE + 6)
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        recs = pool.map(_one, specs, chunksize=1)
    json.dump({"seed": gen.SEED_BASE + 6, "pool_size": pool_size, "records": recs},
              open(OUT, "w"), indent=0)
    print(OUT, len(recs), "records")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 128)
