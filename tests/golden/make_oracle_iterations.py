"""Write tests/golden/oracle_iterations.json: the oracle's per-timestep Newton iteration counts on
the 50x50 single-fracture case and on the 400x400 matrix + 300-segment DFN case, for standard
Newton (mode 0) and Algorithm 1 (mode 1), at the operating tolerance (tol_dp = eps_p = 0.3 psi,
CNV < 1e-6) and at a tight tolerance (tol_dp = 1 Pa, CNV < 1e-10).

Also records:
- at the operating tolerance, the largest difference between the final fields of the two methods
  (max |p_loc - p_std| in psi, max |Sw_loc - Sw_std|): the localized method drops updates below
  eps_p outside its active set, so the two discrete solutions differ by a few cutoffs;
- at the tight tolerance, standard Newton's final p and Sw at 2,000 seeded sample cells and at the
  well cells (17 significant digits), the reference for the GPU's standard Newton on the large case.

Calls only the oracle (plain C, FP64, hand-written sparse LU).  Standard Newton on the 166,659-cell
case factors the whole Jacobian every iteration and takes about 40 minutes on one core, which is
why its results are stored instead of recomputed by the tests.  The runs go to separate processes.

    python tests/golden/make_oracle_iterations.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RUNS = {
    "operating": dict(),
    "tight": dict(tol_dp=1.0, tol_cnv=1e-10, max_newton=40),
}
N_SAMPLES = 2000


def sample_cells(case):
    import numpy as np

    rng = np.random.default_rng(0)
    cells = rng.choice(case.n, min(N_SAMPLES, case.n), replace=False)
    return sorted(set(int(c) for c in cells) | set(int(c) for c in case.well_cell))


def _job(args):
    name, run, mode = args
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2008_01539_gb300 import casegen as cg

    case = getattr(cg, name)()
    t = time.time()
    sim = O.Sim(case, O.Options(mode=mode, **RUNS[run]))
    st = sim.run(case.dt_schedule)
    out = {"status": [int(s["status"]) for s in st], "iterations": [int(s["iterations"]) for s in st],
           "cell_updates": int(sum(s["cell_updates"] for s in st)), "seconds": round(time.time() - t, 1)}
    print(name, run, mode, out["seconds"], sum(out["iterations"]), flush=True)
    return (name, f"{run}_mode{mode}"), out, sim.p.copy(), sim.sw.copy()


def main():
    from paper_2008_01539_gb300 import casegen as cg

    jobs = [(name, run, mode) for name in ("config1", "config0") for run in RUNS for mode in (0, 1)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        results = pool.map(_job, jobs, chunksize=1)
    out = {"description": __doc__.strip().splitlines()[0], "cases": {}}
    for name in ("config0", "config1"):
        case = getattr(cg, name)()
        res = {"n_cells": int(case.n), "timesteps": int(len(case.dt_schedule))}
        final = {}
        for (nm, key), r, p, sw in results:
            if nm == name:
                res[key] = r
                final[key] = (p, sw)
        (p0, s0), (p1, s1) = final["operating_mode0"], final["operating_mode1"]
        res["operating_max_abs_dp_psi_loc_vs_std"] = float(abs(p1 - p0).max() / cg.PSI)
        res["operating_max_abs_dsw_loc_vs_std"] = float(abs(s1 - s0).max())
        cells = sample_cells(case)
        pt, swt = final["tight_mode0"]
        res["tight_mode0_samples"] = {"cells": cells, "p": [float(repr(float(pt[c]))) for c in cells],
                                      "sw": [float(repr(float(swt[c]))) for c in cells]}
        out["cases"][name] = res
    with open(os.path.join(HERE, "oracle_iterations.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
