"""Write sgp_horizon.json: how far the FP64 oracle's own SGP run moves when the data move by 1e-7.

    python tests/golden/make_sgp_horizon.py

Calls only the oracle (and the seeded scene generator).  The 256^2 star field (50 stars, Gaussian
PSF sigma = 2, b = 10, seed 0) is run for 200 SGP iterations from the exact float32 data and from
eight copies whose counts are multiplied by 1 + 1e-7 n (n standard normal, seeds 1..8): the FP32
rounding level of the data.  The relative KL differences after 200 iterations bound what any
FP32 implementation can be asked to match (Sect. 3.2 parameters, Algorithm 1).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import sgp_oracle as O               # noqa: E402
from paper_1210_2258_b300 import scenes          # noqa: E402


def problem(sc):
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return O.Problem(f32(sc.psfs), f32(sc.g), f32(sc.b))


def main():
    sc = scenes.stars_scene(seed=0, N=256)
    n = 200
    ref = O.sgp(problem(sc), stop=O.StopRule("fixed", n))
    out = {"source": __doc__.strip().splitlines()[0], "scene": "stars_scene(seed=0, N=256)", "iterations": n,
           "J_ref": ref.J, "perturbation": 1e-7, "runs": []}
    for s in range(1, 9):
        p = problem(sc)
        p.g = p.g * (1 + 1e-7 * np.random.default_rng(s).standard_normal(p.g.shape))
        r = O.sgp(p, stop=O.StopRule("fixed", n))
        out["runs"].append({"seed": s, "J": r.J, "rel_J": abs(r.J - ref.J) / ref.J,
                            "rel_f": float(np.linalg.norm(r.f - ref.f) / np.linalg.norm(ref.f))})
    out["max_rel_J"] = max(r["rel_J"] for r in out["runs"])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "sgp_horizon.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "runs"}))


if __name__ == "__main__":
    main()
