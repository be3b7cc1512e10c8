"""Write the oracle's stored results under tests/golden/ (run on the CPU).

This script imports only ``oracle`` (the FP64 CPU oracle) and ``bte_inputs``
(the seeded synthetic workloads); no value it stores comes from the CUDA
library.  The GPU parity tests compare libbte against these files:

* ``hotspot64_k20.npz``: T after exactly 20 source iterations of the full
  64^3 hotspot (15 bands x 128 directions, Gaussian source) from T = 300 K;
* ``finfet_k20.npz``: the same for the full 160x80x64 FinFET (solid cells);
* ``finfet_s2_adjoint.npz``: the FinFET at half resolution (80x40x32, all 15
  bands x 128 directions) converged to eps_T < 1e-8, its iteration count and
  T, and the discrete-adjoint gradients (tau_b, T_sub, Q_amp) of the probe
  misfit J = 1/2 sum_p (T_p - T_obs,p)^2, with T_obs from a truth run with
  tau_b x 1.2, T_sub = 301 K and Q x 0.8.

    python tests/golden/make_goldens.py [hotspot] [finfet] [finfet_s2]

Each job runs in a process of its own (spawned, so no state is shared); the
half-resolution FinFET's truth run is a job of its own that runs next to
its solve and hands the probe temperatures over through a temporary file.
The full-size jobs hold e and its previous iterate in FP64 (about 8 GB for
the hotspot, 25 GB for the FinFET).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def _setup():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def job_hotspot():
    _setup()
    import bte_inputs as bi
    import oracle
    p = bi.hotspot_3d()
    t0 = time.time()
    r = oracle.solve(p, max_iter=20, tol=0.0)
    np.savez_compressed(os.path.join(HERE, "hotspot64_k20.npz"), T=r["T"], iters=r["iters"],
                        eps=r["eps"])
    return f"hotspot k=20: {time.time() - t0:.0f} s"


def job_finfet():
    _setup()
    import bte_inputs as bi
    import oracle
    p = bi.finfet_3d()
    t0 = time.time()
    r = oracle.solve(p, max_iter=20, tol=0.0)
    act = np.flatnonzero(p.mask)
    np.savez_compressed(os.path.join(HERE, "finfet_k20.npz"), cells=act.astype(np.int32), T=r["T"][act],
                        iters=r["iters"], eps=r["eps"])
    return f"finfet k=20: {time.time() - t0:.0f} s"


TRUTH_S2 = os.path.join(HERE, "_finfet_s2_truth.npz")   # passed between the two half-resolution jobs


def job_finfet_s2_truth():
    """The truth run of the half-resolution FinFET (its probe temperatures),
    in a process of its own next to the solve of job_finfet_s2."""
    _setup()
    import bte_inputs as bi
    import oracle
    t0 = time.time()
    p = bi.finfet_3d(scale=2)
    truth = bi.finfet_3d(scale=2, tau_b_scale=1.2, T_sub=301.0, Q_amp=0.8e19)
    rt = oracle.solve(truth, max_iter=100000, tol=1e-8)
    probes = np.asarray(p.probes)
    tmp = TRUTH_S2 + ".tmp.npz"
    np.savez(tmp, T_obs=rt["T"][probes], iters=rt["iters"])
    os.replace(tmp, TRUTH_S2)
    return f"finfet s2 truth ({rt['iters']} it): {time.time() - t0:.0f} s"


def job_finfet_s2():
    _setup()
    import bte_inputs as bi
    import oracle
    t0 = time.time()
    p = bi.finfet_3d(scale=2)
    probes = np.asarray(p.probes)
    r = oracle.solve(p, max_iter=100000, tol=1e-8)
    # the truth run's probe temperatures (job_finfet_s2_truth)
    while not os.path.exists(TRUTH_S2):
        time.sleep(10.0)
    with np.load(TRUTH_S2) as tr:
        T_obs = tr["T_obs"].copy()
        rt = {"iters": int(tr["iters"])}
    os.remove(TRUTH_S2)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, r["T"][probes] - T_obs)
    a = oracle.adjoint(p, r["e"], r["T"], g, max_iter=100000, tol=1e-10)
    np.savez_compressed(os.path.join(HERE, "finfet_s2_adjoint.npz"), T=r["T"], iters=r["iters"],
                        probes=probes, T_obs=T_obs, g_tau=a["g_tau"], g_Tw=a["g_Tw"], g_Q=a["g_Q"],
                        adj_iters=a["iters"], truth_iters=rt["iters"])
    return f"finfet s2 converged ({r['iters']} it) + adjoint ({a['iters']} it): {time.time() - t0:.0f} s"


JOBS = {"hotspot": job_hotspot, "finfet": job_finfet, "finfet_s2": job_finfet_s2,
        "finfet_s2_truth": job_finfet_s2_truth}


def _run(name):
    return JOBS[name]()


if __name__ == "__main__":
    names = sys.argv[1:] or ["hotspot", "finfet", "finfet_s2"]
    if "finfet_s2" in names and "finfet_s2_truth" not in names:
        names.append("finfet_s2_truth")   # its truth run, in parallel
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(names)) as pool:
        for msg in pool.imap_unordered(_run, names):
            print(msg, flush=True)
