"""Write the oracle regression fixtures in this folder.

Calls only the CPU oracle (``oracle/``) on seeded ``synth`` inputs; nothing here
comes from the GPU library.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def cases():
    """(name, model, f) triples; f is a seeded uniform draw over the window states."""
    out = []
    for name, m in (("tiny4", synth.make_tiny(4)), ("window12", synth.make_window4(12))):
        o = oracle.Oracle(m)
        f = np.random.default_rng(20251103).uniform(0.0, 1.0, o.nstate)
        out.append((name, m, f))
    return out


def main():
    for name, m, f in cases():
        o = oracle.Oracle(m)
        I = o.collision(f)
        r = o.rates(f)
        path = os.path.join(HERE, f"oracle_{name}.txt")
        with open(path, "w") as fh:
            fh.write(f"# oracle regression fixture: {name}, nstate={o.nstate}, channels={o.count_channels()}\n")
            fh.write("# f = numpy default_rng(20251103).uniform(0,1,nstate); columns: f, I (1/fs), 1/tau (1/fs)\n")
            for a, b, c in zip(f, I, r):
                fh.write(f"{a:.17e} {b:.17e} {c:.17e}\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
