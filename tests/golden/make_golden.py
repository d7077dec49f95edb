"""Write the stored expected values of the dual ascent (calls only oracle/).

For each named workload the oracle runs the full iteration count and records
LB after every pass plus order-sensitive hashes of the exported state
(x = B, y = C, z = D in the compact layouts of include/rlt2.h) after selected
passes.  Usage: python tests/golden/make_golden.py [workload ...]
       python tests/golden/make_golden.py --f64 [workload ...]   (FP64 form)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_1510_02065_gb300 import instances        # noqa: E402
from tests.layout import compact_y, compact_z, state_hash  # noqa: E402

HASH_AT = {1, 2, 3, 5, 10, 20, 50, 100, 150, 200, 300}


def make(name):
    F, D, iters = instances.instance(name)
    st = O.State(F, D)
    lb, hashes = [], {}
    t0 = time.time()
    for t in range(1, iters + 1):
        lb.append(st.iterate())
        if t in HASH_AT or t == iters:
            hashes[str(t)] = dict(x=state_hash(st.b), y=state_hash(compact_y(st.c)),
                                  z=state_hash(compact_z(st.d)))
    out = dict(workload=name, N=int(F.shape[0]), iters=iters, lb=lb, hash=hashes,
               work=st.work(), oracle_seconds=round(time.time() - t0, 1),
               generated_by="tests/golden/make_golden.py (oracle/ only)")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lb_%s.json" % name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(name, "LB", lb[0], "->", lb[-1], "in %.1fs" % out["oracle_seconds"])


def bits(a):
    """Bit patterns of doubles as int64 (so that hashes and JSON are exact)."""
    import numpy as np
    return np.ascontiguousarray(a, np.float64).view(np.int64)


def make_f64(name):
    """The same record for the FP64 form (reading R14): LB as the int64 bit
    patterns of the doubles, state hashes over the bit patterns."""
    F, D, iters = instances.instance(name)
    st = O.StateF64(F, D)
    lb, hashes = [], {}
    t0 = time.time()
    for t in range(1, iters + 1):
        lb.append(int(bits([st.iterate()])[0]))
        if t in HASH_AT or t == iters:
            hashes[str(t)] = dict(x=state_hash(bits(st.b)), y=state_hash(bits(compact_y(st.c))),
                                  z=state_hash(bits(compact_z(st.d))))
    out = dict(workload=name, N=int(F.shape[0]), iters=iters, form="fp64", lb_bits=lb, hash=hashes,
               work=st.work(), oracle_seconds=round(time.time() - t0, 1),
               generated_by="tests/golden/make_golden.py --f64 (oracle/ only)")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lb_f64_%s.json" % name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(name, "FP64 in %.1fs" % out["oracle_seconds"])


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "--f64":
        for name in args[1:] or ["clustered_n20"]:
            make_f64(name)
    else:
        for name in args or ["uniform_n8", "grid_n12", "clustered_n20"]:
            make(name)
