"""Write workloads/critical_masses.json: near-critical masses of the benchmark
gauge configurations, computed by the oracle's critical-mass finder only.

Test infrastructure (see ``oracle/__init__.py``): the stored masses are inputs
of the workloads; every value in the file comes from ``oracle.critical``.
Each entry also records the mean plaquette and Q of the configuration so that
a regenerated configuration can be checked against it.

    python -m oracle.find_critical_masses [--out FILE] [name ...]

The configurations of the serving workload are written to
workloads/critical_masses_serving.json (``--out``).
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W                       # noqa: E402
from oracle import critical                 # noqa: E402

OUT = os.path.join(ROOT, "workloads", "critical_masses.json")

# name -> (L, beta, sweeps, seed)
CONFIGS = {
    "L128_b6_s1": (128, 6.0, 200, 1),
    "L128_b6_s2": (128, 6.0, 200, 2),
    "L256_b10_s1": (256, 10.0, 500, 1),
    "L1024_b10_s1": (1024, 10.0, 500, 1),
    # serving workload: 64^2 beta 3, 128^2 beta 6, 256^2 and 512^2 beta 10, two seeds each
    "L64_b3_s1": (64, 3.0, 200, 1),
    "L64_b3_s2": (64, 3.0, 200, 2),
    "L256_b10_s2": (256, 10.0, 500, 2),
    "L512_b10_s1": (512, 10.0, 500, 1),
    "L512_b10_s2": (512, 10.0, 500, 2),
}


def main(names, out=OUT):
    for name in names:
        L, beta, sweeps, seed = CONFIGS[name]
        tried = []
        while True:
            t0 = time.time()
            th = W.quenched_u1_angles(L, L, beta, sweeps, seed)
            res = critical.near_critical_mass(W.links_from_angles(th))
            tried.append(seed)
            if res is not None:
                break
            seed += 1000                    # no real mode near the physical branch
        res.update({"L": L, "beta": beta, "sweeps": sweeps, "seed": seed, "seeds_tried": tried,
                    "plaquette": W.mean_plaquette(th), "Q": round(W.topological_charge(th)),
                    "finder_seconds": round(time.time() - t0, 1)})
        print(name, res, flush=True)
        data = json.load(open(out)) if os.path.exists(out) else {}   # re-read: other runs may write
        data[name] = res
        json.dump(data, open(out, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    out = OUT
    if args[:1] == ["--out"]:
        out, args = os.path.join(ROOT, args[1]) if not os.path.isabs(args[1]) else args[1], args[2:]
    main(args or list(CONFIGS), out)
