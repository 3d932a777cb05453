"""Record the oracle's own block-CG iteration counts for the benchmark chips.

Writes oracle/recorded_iterations.json.  Only the oracle and the seeded input
generator run here.  The benchmark's CPU-baseline leg times a bounded sample
of oracle iterations and scales it by these counts.

    python oracle/record_iterations.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import blockoa_oracle as orc  # noqa: E402
from paper_2510_23221_gb300 import synth  # noqa: E402


def main():
    out = {}
    for name, w, rtol in (("chip128x128x8_s32", synth.single_chip_workload(M=1), 1e-6),
                          ("chip32x32x4_s8", synth.small_fp64_workload(M=1), 1e-12)):
        chip = w.chips[0]
        A = orc.assemble(chip)
        B = orc.rhs(chip, w.density[0])
        t = time.perf_counter()
        _, info = orc.block_cg(A, B, rtol=rtol, maxiter=100000)
        out[name] = {"rtol": rtol, "iters": int(info["iters"]), "status": int(info["status"]),
                     "relres_max": float(info["relres"].max()),
                     "seconds_here": round(time.perf_counter() - t, 2)}
        print(name, out[name])
    with open(os.path.join(HERE, "recorded_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
