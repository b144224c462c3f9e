"""Writes tests/golden/astar_full_size.json: a* of the full-size workloads computed by the FP64 oracle only
(C-PCG, Jacobi, tolerance 1e-13), for the GPU tests that cannot afford the oracle at run time:
cfg2 and cfg4 (one instance each), cfg3 (all 64 instances of the batched workload, in instance order), and
cfg4_half (cfg4 on the Nyquist-free modes: oracle homogenized_nyquist_free, the half-spectrum plans' scheme).

Run from the repository root: python tests/golden/make_golden.py [cfg2] [cfg3] [cfg4] [cfg4_half]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import qp_workloads as W  # noqa: E402
from oracle import qp_oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "astar_full_size.json")
HOW = "oracle/qp_oracle.py homogenized(tol=1e-13), Jacobi C-PCG (Algorithm 2)"


def one(inst, nyquist_free=False):
    t0 = time.time()
    solve = O.homogenized_nyquist_free if nyquist_free else O.homogenized
    A, Us, infos, Ac = solve(inst, tol=1e-13)
    rec = {"name": inst.name, "astar_re": A.tolist(), "astar_im": Ac.imag.tolist(),
           "iterations": [i["iterations"] for i in infos],
           "rel_residual": [i["rel_residual"] for i in infos],
           "oracle_seconds": round(time.time() - t0, 1),
           "how": HOW.replace("homogenized(", "homogenized_nyquist_free(") if nyquist_free else HOW}
    if "clamped_fraction" in inst.meta:
        rec["clamped_fraction"] = inst.meta["clamped_fraction"]
    print(inst.name, A.tolist(), [i["iterations"] for i in infos], rec["oracle_seconds"], flush=True)
    return rec


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        if name == "cfg3":
            data[name] = {"instances": [one(inst) for inst in W.cfg3()], "how": HOW}
        elif name.endswith("_half"):
            data[name] = one(getattr(W, name[:-5])(), nyquist_free=True)
        else:
            data[name] = one(getattr(W, name)())
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["cfg2", "cfg3", "cfg4"])
