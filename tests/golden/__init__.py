"""Values printed in the paper, read from the text fixtures beside this file.

Each fixture line is ``name = value ; citation ; description``; only values
the paper prints go here (nothing computed by either implementation)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def _load(fname):
    out = {}
    with open(os.path.join(_HERE, fname)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, cite, _ = (s.strip() for s in line.split(";", 2))
            name, val = (s.strip() for s in head.split("=", 1))
            if not cite:
                raise ValueError(f"{fname}: {name} has no citation")
            out[name] = float(val)
    return out


PAPER = _load("paper_values.txt")
