"""Write the long-trajectory fixtures in this folder: the oracle's own rt-BTE trajectory.

Classic RK4 on df/dt = I[f] (Eq. 1 with no field, Eq. 2 for I) with dt = 1 fs from the hot
Gaussian population, computed by the CPU oracle (``oracle/``) on seeded ``synth`` inputs only;
nothing here comes from the GPU library.  Two workloads:

* ``window24``: 24^3 grids, 4 bands, 6 modes (1028 states): f after 250, 500, 750 and 1000
  steps;
* ``window40``: the 40^3 workload (4756 states): f after 50 steps.

Run from the repository root (it takes minutes on a few cores):

    python tests/golden/make_trajectory.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = {"window24": (250, 4), "window40": (50, 1)}  # steps per checkpoint, checkpoints


def write(name):
    every, nck = CASES[name]
    m = synth.make_config(name)
    o = oracle.Oracle(m)
    f = o.window_values(m.f_hot())
    cols = []
    t0 = time.time()
    for _ in range(nck):
        f = o.rk4(f, 1.0, every)
        cols.append(f.copy())
    path = os.path.join(HERE, f"trajectory_{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# oracle rt-BTE trajectory: {name}, nstate={o.nstate}, classic RK4, dt = 1 fs, from the hot "
                 f"population (synth f_hot)\n")
        fh.write("# columns: f after " + ", ".join(str(every * (k + 1)) for k in range(nck)) + " steps\n")
        for r in range(o.nstate):
            fh.write(" ".join(f"{c[r]:.17e}" for c in cols) + "\n")
    print(f"wrote {path} ({time.time() - t0:.0f} s)")


def main():
    for name in (sys.argv[1:] or list(CASES)):
        write(name)


if __name__ == "__main__":
    main()
