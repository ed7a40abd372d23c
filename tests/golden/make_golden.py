"""Write the oracle's results for the full-length benchmark runs into tests/golden/.

Calls only the FP64 oracle (oracle/) and the input generators.  For each workload it stores the
observables after the full run (mass, ||E_phi||_2 of Eq. err, max/min phi) and the oracle's phi at a
seeded sample of nodes (half of them drawn from the interface region 0.02 < phi0 < 0.98), and for the
translation and Zalesak workloads the whole final field (<name>_phi.npz), so the GPU path can be checked at
full length, at every node, without rerunning the oracle.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1805_00007_gb300 import workloads as wl  # noqa: E402


def sample_nodes(phi0, n, seed):
    rng = np.random.default_rng(seed)
    ny, nx = phi0.shape
    flat = np.arange(nx * ny)
    iface = flat[((phi0 > 0.02) & (phi0 < 0.98)).ravel()]
    a = rng.choice(iface, size=min(n // 2, iface.size), replace=False)
    b = rng.choice(flat, size=n - a.size, replace=False)
    idx = np.unique(np.concatenate([a, b]))
    return idx // nx, idx % nx


def make(name, p, phi0, nsteps, seed, full_field=False):
    t = time.time()
    phi, _ = oracle.simulate(p, phi0, nsteps)
    ob = oracle.observe(phi, phi0)
    j, i = sample_nodes(phi0, 2048, seed)
    out = {"workload": name, "params": p, "nsteps": nsteps, "generator": "tests/golden/make_golden.py (oracle only)",
           "mass0": float(phi0.sum()), "mass": ob["mass"], "err_l2": ob["err_l2"], "max": ob["max"],
           "min": ob["min"], "nodes_j": j.tolist(), "nodes_i": i.tolist(), "phi": phi[j, i].tolist()}
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(out, fh)
    if full_field:
        # the whole final field, so that a check can compare every node (about 7 bytes per node compressed)
        np.savez_compressed(os.path.join(HERE, f"{name}_phi.npz"), phi=phi, nsteps=nsteps)
    print(name, f"{time.time() - t:.1f}s", {k: out[k] for k in ("err_l2", "max", "min")}, flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["translation_100", "zalesak_256", "vortex_512"]
    if "translation_100" in which:
        p, phi0, T = wl.translation()
        make("translation_100", p, phi0, T, 1, full_field=True)
    if "zalesak_256" in which:
        p, phi0, T = wl.zalesak()
        make("zalesak_256", p, phi0, T, 2, full_field=True)
    if "vortex_512" in which:
        p, phi0, T = wl.single_vortex()
        make("vortex_512", p, phi0, T, 3)
