"""Write tests/golden/c3_oracle_sigma.json: the FP64 oracle's singular values
after each of the first 23 add-rows batches of C3 (users x items ratings,
1,000,000 x 50,000, Zipf 1.1 item popularity, ~20 ratings per user, k = 128,
users appended in batches of s = 1024 from a start on the first 500,000
users; the start uses 2 power iterations).  Calls only synth/ and oracle/
(the sparse method, Algorithm 11).  Run: python tests/golden/make_c3_oracle_sigma.py
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import synth  # noqa: E402
from oracle import svlcov  # noqa: E402

N_BATCHES = 23


def main():
    t0 = time.time()
    p = synth.c3_problem(n_batches=N_BATCHES, power_iters=2)
    t1 = time.time()
    st = svlcov.State.init(p["U"], p["sigma"], p["V"])
    per_batch = []
    for kind, b in p["batches"]:
        st.apply(kind, b)
        per_batch.append(st.sigma.tolist())
    out = dict(
        source="FP64 oracle (oracle.svlcov.State, Algorithms 2 and 11) on synth.c3_problem(n_batches=23, "
               "power_iters=2)",
        workload="C3 ratings: 1e6 users x 5e4 items, Zipf 1.1, k=128, add_rows batches of s=1024",
        sigma_initial=p["sigma"].tolist(), sigma_after_batch=per_batch, resets=st.resets,
        seconds_generation=t1 - t0, seconds_oracle=time.time() - t1)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle_sigma.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, "in", time.time() - t0, "s")


if __name__ == "__main__":
    main()
