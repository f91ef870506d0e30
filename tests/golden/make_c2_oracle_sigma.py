"""Write tests/golden/c2_oracle_sigma.json: the FP64 oracle's singular values
after every node batch of the full C2 trajectory (graph node insertion,
Chung-Lu N = 100000, k = 64, s = 256, rows then columns per node batch), so
that a benchmark run of any length can be compared with the oracle at the
node batch where it stops.  Calls only synth/ and oracle/ (the sparse method
of Algorithms 2, 3 and 11).  Run: python tests/golden/make_c2_oracle_sigma.py
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import svlcov  # noqa: E402


def main():
    t0 = time.time()
    p = synth.c2_problem()
    st = svlcov.State.init(p["U"], p["sigma"], p["V"])
    per_batch = []
    for i, (kind, b) in enumerate(p["batches"]):
        st.apply(kind, b)
        if kind == "cols":
            per_batch.append(st.sigma.tolist())
    out = dict(
        source="FP64 oracle (oracle.svlcov.State, Algorithms 2, 3, 11) on synth.c2_problem() defaults",
        workload="C2 graph node insertion: Chung-Lu N=100000, gamma=2.1, mean degree 10, k=64, s=256",
        n_node_batches=len(p["batches"]) // 2, mean_degree=p["mean_degree"],
        sigma_initial=p["sigma"].tolist(), sigma_after_node_batch=per_batch, sigma_final=st.sigma.tolist(),
        resets=st.resets, seconds=time.time() - t0)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_sigma.json")
    with open(path, "w") as f:
        # one line per array keeps the file small and diffable
        f.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in out.items()) + "\n}\n")
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
