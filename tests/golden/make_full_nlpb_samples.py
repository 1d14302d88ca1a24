"""Writes sampled potentials of the full-size nonlinear Poisson-Boltzmann
workloads, computed by the oracle alone, as small text fixtures.

Each fixture holds the oracle's Algorithm 4 result (Newton inner operator,
the linear PB term of Eq. corrPB at the current potential; Eisenstat-Walker
choice-2 forcing from 0.3; outer residual in charge units below 1e-11) on
the seeded synthetic inputs of one workload:
  surface_nlpb_160x160x256.txt  surface BC slab, 160 x 160 x 256, 0.1 M
  free_nlpb_256.txt             free BC 256^3, 200 charges in a union of
                                spheres, 0.5 M
with the whole field's L2 norm, maximum magnitude and sum, and the values at
2048 seeded flat indices plus the index of the largest magnitude.  The full
fields (52 MB and 134 MB) are too large to store; the GPU tests compare
their own full-size results at these indices.

    python tests/golden/make_full_nlpb_samples.py [surface|free ...]

The free 256^3 solve takes about an hour on eight cores."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

TOL = 1e-11
FORCING = 0.3
SAMPLES = 2048
CASES = {
    "surface": (3, "surface_nlpb_160x160x256.txt",
                "surface BC slab 160 x 160 x 256 (seeded workload 3), nonlinear PB at 0.1 M"),
    "free": (4, "free_nlpb_256.txt",
             "free BC 256^3, 200 charges in a union-of-spheres cavity (seeded workload 4), nonlinear PB at 0.5 M"),
}


def sample_indices(size, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(size, SAMPLES, replace=False))


def make(name):
    wl, fname, what = CASES[name]
    p = synth.workload(wl, kind="nlpb")
    t0 = time.time()
    phi, info = oracle.solve_nlpb(p.grid, p.rho, p.eps, p.electrolyte, p.eps0, tol=TOL, max_iter=4000,
                                  forcing=FORCING, forcing_rule="ew2")
    if not info["converged"]:
        raise SystemExit(f"{name}: oracle did not converge")
    flat = phi.ravel()
    idx = sample_indices(flat.size, 20150900 + wl)
    amax = int(np.argmax(np.abs(flat)))
    idx = np.unique(np.append(idx, amax))
    lines = [
        f"# {what}",
        "# oracle Algorithm 4: Newton inner operator (linear PB term of Eq. corrPB at the current potential),",
        f"# Eisenstat-Walker choice-2 forcing from {FORCING}, outer residual (charge units) <= {TOL:g}",
        "# written by: python tests/golden/make_full_nlpb_samples.py " + name,
        f"shape {' '.join(str(s) for s in p.grid.shape)}",
        f"outer {info['outer']} inner {int(sum(info['inner']))} seconds {time.time() - t0:.0f}",
        f"l2 {np.sqrt(np.sum(flat * flat)):.17e}",
        f"maxabs {np.max(np.abs(flat)):.17e} at {amax}",
        f"sum {np.sum(flat):.17e}",
    ]
    lines += [f"{i} {flat[i]:.17e}" for i in idx]
    with open(os.path.join(HERE, fname), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(name, lines[5], flush=True)


def load(fname):
    """Parses a fixture: (shape, {'l2','maxabs','sum'}, indices, values)."""
    shape, stats, idx, val = None, {}, [], []
    with open(os.path.join(HERE, fname)) as f:
        for line in f:
            if line.startswith("#"):
                continue
            w = line.split()
            if w[0] == "shape":
                shape = tuple(int(x) for x in w[1:])
            elif w[0] in ("l2", "maxabs", "sum"):
                stats[w[0]] = float(w[1])
            elif w[0] == "outer":
                continue
            else:
                idx.append(int(w[0]))
                val.append(float(w[1]))
    return shape, stats, np.array(idx, dtype=np.int64), np.array(val)


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["surface", "free"]):
        make(n)
