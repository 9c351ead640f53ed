"""Write workloads/oracle_iterations.json: the oracle's MG-CG iteration counts
and per-phase CPU times on each benchmark workload (one thread).

Test infrastructure (see ``oracle/__init__.py``); every stored value comes
from the oracle.  The benchmark's CPU reference leg times a bounded sample of
the oracle and scales it to whole solves with these counts.

    python -m oracle.workload_iterations [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W                        # noqa: E402
from oracle import krylov, multigrid, wilson  # noqa: E402

OUT = os.path.join(ROOT, "workloads", "oracle_iterations.json")


def run(name):
    wl = W.BENCH_WORKLOADS[name]
    crit = json.load(open(os.path.join(ROOT, "workloads", "critical_masses.json")))[wl["critical_key"]]
    U = W.quenched_u1(wl["Lx"], wl["Lt"], wl["beta"], wl["sweeps"], wl["seed"])
    noise = W.setup_noise(wl["Lx"], wl["Lt"], wl["blocks"], wl["Nv"], wl["noise_seed"])
    chi = W.gaussian_field((wl["Lt"], wl["Lx"], 2), wl["chi_seed"])
    out = {"masses": {}}
    t0 = time.time()
    H = multigrid.setup(U, crit["m_nc"], wl["blocks"], wl["Nv"], noise, sweeps=wl["setup_sweeps"])
    out["setup_seconds"] = round(time.time() - t0, 2)
    for m in [crit["m_nc"]] + list(wl["heavy_masses"]):
        t0 = time.time()
        if m != crit["m_nc"]:
            multigrid.set_mass(H, m)
        t1 = time.time()
        b = wilson.apply_D(U, m, chi, dagger=True)
        x, it, info = krylov.mgcg(H, b, wl["tol"], 20000)
        out["masses"][repr(m)] = {"iterations": it, "true_residual": info["true_res"],
                                  "set_mass_seconds": round(t1 - t0, 2),
                                  "solve_seconds": round(time.time() - t1, 2)}
        print(name, m, out["masses"][repr(m)], flush=True)
    return out


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = run(name)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(W.BENCH_WORKLOADS))
