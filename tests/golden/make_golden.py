"""Write the oracle's reference results for full-size workloads.

Calls only the scene generator and the FP64 CPU oracle (oracle/).  The
stored values let the GPU tests check full-size solves without rerunning the
oracle (about 4 minutes for the driving workload on 8 cores).

    python tests/golden/make_golden.py driving
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2510_15271_b300 import scenes  # noqa: E402

OUTLIER_PX = 5.0
REFINE_MAX, REFINE_TOL = 5, 1e-6   # the city recipe's refinement (reading C11)


def golden(name, seed):
    s = scenes.make_scene(name, seed=seed)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    st = O.state_from_qt(s.cam_qt, s.pts)
    t0 = time.time()
    refine_max = REFINE_MAX if s.refine else 0
    res = O.lm_solve(prob, st, O.LMOptions(huber_delta=s.huber_delta, lm_iters=s.lm_iters,
                                           solver=s.solver, pcg_tol=s.pcg_tol,
                                           pcg_max_iters=s.pcg_max_iters, refine_max=refine_max,
                                           refine_tol=REFINE_TOL))
    dt = time.time() - t0
    return {
        "workload": name, "seed": seed, "n_cams": s.n_cams, "n_pts": s.n_pts, "n_obs": s.n_obs,
        "lm_iters": s.lm_iters, "solver": s.solver, "huber_delta": s.huber_delta,
        "pcg_tol": s.pcg_tol, "pcg_max_iters": s.pcg_max_iters,
        "refine_max": refine_max, "refine_tol": REFINE_TOL,
        "costs": res.costs.tolist(), "accepted": res.accepted.astype(int).tolist(),
        "pcg_iters": res.pcg_iters.tolist(),
        "rmse_all_px": O.rmse(prob, res.state),
        "rmse_inlier_px": O.rmse(prob, res.state, s.obs_inlier),
        "rmse_inlier_trimmed_px": O.rmse(prob, res.state, s.obs_inlier, OUTLIER_PX),
        "outlier_threshold_px": OUTLIER_PX,
        "oracle_seconds": dt,
        "how": "oracle.lm_solve on scenes.make_scene(workload, seed) with its solve settings",
        # final poses (qw, qx, qy, qz, tx, ty, tz; world -> camera), for the
        # pose error of the GPU results against the oracle
        "cam_qt": [[float(v) for v in row] for row in O.state_to_qt(res.state)],
    }


if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "driving"
    seed = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    out = golden(name, seed)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_seed{seed}_oracle.json")
    poses = out.pop("cam_qt")
    text = json.dumps(out, indent=1)
    # one pose per line keeps the file readable and diffable
    text = text[:-2] + ',\n "cam_qt": [\n' + ",\n".join(
        "  " + json.dumps(p) for p in poses) + "\n ]\n}\n"
    with open(path, "w") as f:
        f.write(text)
    print(path, out["rmse_inlier_trimmed_px"], out["oracle_seconds"])
