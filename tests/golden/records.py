"""Stored oracle results for runs too long to repeat in every GPU test
session: the grid centres, time, norm, energy, the discrete L2 norm of psi
and psi itself at 1024 grid points (the 512 of largest modulus and 512 drawn
from a seeded generator).  Written by the make_*.py scripts beside this file,
which call only the oracle; read by the GPU tests."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def sample_indices(psi, seed):
    from tests import inputs

    flat = np.abs(psi.ravel())
    top = np.argsort(flat)[::-1][:512]
    rest = np.setdiff1d(np.arange(flat.size), top)
    rnd = inputs.rng(seed).choice(rest, 512, replace=False)
    return np.sort(np.concatenate([top, rnd]))


def write(path, o, title, seconds, seed):
    psi, q, p, t = o.get_state()
    n, E, _, _ = o.observables()
    flat = psi.ravel()
    idx = sample_indices(psi, seed)
    with open(path, "w") as f:
        f.write(f"# FP64 oracle: {title}\n")
        f.write(f"# written by tests/golden/{os.path.basename(__import__('sys').argv[0])} "
                f"({seconds:.0f} s of oracle time)\n")
        f.write("q = " + " ".join(repr(float(v)) for v in q) + "\n")
        f.write("p = " + " ".join(repr(float(v)) for v in p) + "\n")
        f.write(f"t = {t!r}\n")
        f.write(f"norm = {n!r}\n")
        f.write(f"energy = {E!r}\n")
        f.write(f"psi_l2 = {float(np.linalg.norm(flat))!r}\n")
        for i in idx:
            f.write(f"{int(i)} {float(flat[i].real)!r} {float(flat[i].imag)!r}\n")


def read(name):
    """dict with q, p (arrays), t, norm, energy, psi_l2 and idx, psi (samples)."""
    rec, idx, vals = {}, [], []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if "=" in line:
                k, v = (s.strip() for s in line.split("=", 1))
                nums = [float(x) for x in v.split()]
                rec[k] = np.array(nums) if k in ("q", "p") else nums[0]
            else:
                i, re, im = line.split()
                idx.append(int(i))
                vals.append(complex(float(re), float(im)))
    rec["idx"] = np.array(idx, dtype=np.int64)
    rec["psi"] = np.array(vals)
    return rec


def read_scalars(name):
    """dict of the `key = values` lines of a stored record (arrays for
    several values, floats for one)."""
    rec = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#") or "=" not in line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            nums = [float(x) for x in v.split()]
            rec[k] = np.array(nums) if len(nums) > 1 else nums[0]
    return rec
