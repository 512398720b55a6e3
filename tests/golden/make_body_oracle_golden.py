"""Write tests/golden/body_2mm_oracle.json from the CPU oracle alone.

Solves the full-size body phantom (256 x 160 x 896 voxels, h = 2 mm,
9,250,062 unknowns, 0.3 m / 1000 A loop 0.4 m below the phantom) with the
oracle's Jacobi-preconditioned CG twice -- to the 1e-8 relative residual of
the benchmark and to the oracle's 1e-13 -- and records the iteration counts,
residuals, wall times and thread count, plus Psi (zero mean per component)
at 4096 seeded unknowns of the 1e-13 solve and its 2-norm, and the
voxel-averaged |E| of Eq. 1 from that solve at 8192 seeded conducting voxels
with its maximum over the body and the floor scale omega/h * max|a| of the
|E| comparison.  Nothing here touches the CUDA path.  Run from the
repository root:

    python tests/golden/make_body_oracle_golden.py
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from spfd_inputs import body_phantom, loop_potential  # noqa: E402


def main():
    out = os.path.join(ROOT, "tests", "golden", "body_2mm_oracle.json")
    t0 = time.time()
    ph = body_phantom()
    a = loop_potential(ph.dims, ph.h, ph.origin)
    t_in = time.time() - t0
    t0 = time.time()
    sys_ = oracle.assemble(ph.sigma, ph.h)
    b = oracle.project(sys_, oracle.rhs(sys_, a))
    t_asm = time.time() - t0
    rec = {"workload": "body phantom 256x160x896 voxels, h=2 mm, loop R=0.3 m I=1000 A at z=-0.4 m",
           "n_dof": sys_.n, "n_comp": sys_.ncomp, "threads": oracle.num_threads(),
           "inputs_s": t_in, "assemble_s": t_asm}
    for tol in (1e-8, 1e-13):
        t0 = time.time()
        x, info = oracle.pcg(sys_, b, tol=tol, maxit=2_000_000)
        dt = time.time() - t0
        key = "tol_%g" % tol
        rec[key] = {"iters": info["iters"], "rel_res": info["rel_res"],
                    "converged": info["converged"], "wall_s": dt,
                    "s_per_iter": dt / max(info["iters"], 1)}
        print(key, rec[key], flush=True)
    x = oracle.project(sys_, x)
    rng = np.random.default_rng(2010)
    pick = np.sort(rng.choice(sys_.n, size=4096, replace=False))
    rec["psi_sample_nodes"] = sys_.nodes[pick].tolist()
    rec["psi_sample_values"] = x[pick].tolist()
    rec["psi_norm2"] = float(np.linalg.norm(x))
    omega = 2 * np.pi * 85e3
    E = oracle.efield(ph.sigma, a, sys_.scatter(x), ph.h, omega)
    cond = np.flatnonzero(ph.sigma.reshape(-1) > 0)
    vpick = np.sort(np.random.default_rng(12879).choice(cond.size, size=8192, replace=False))
    rec["omega"] = omega
    rec["E_sample_voxels"] = cond[vpick].tolist()
    rec["E_sample_values"] = E.reshape(-1)[cond[vpick]].tolist()
    rec["E_max"] = float(E.max())
    rec["E_floor_scale"] = float(omega / ph.h * np.abs(a).max())
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
