"""Readers of the stored expected values under tests/golden/ (written by
tests/golden/make_golden.py from the oracle only)."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
DIMS = (8, 8, 8, 8)
M0, CSW, EPS, GSEED, PSEED, VSEED = -0.2, 1.0, 0.4, 301, 302, 303


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            out.append([float(v) for v in line.split()])
    return np.array(out)


def site_values(name):
    """{(x, y, z, t, spin, colour): complex} of a site file."""
    r = rows(name)
    return {tuple(int(v) for v in row[:6]): complex(row[6], row[7]) for row in r}


def compare_sites(name, field):
    """max |field - stored| / max |stored| over the stored sites; field (Lt,Lz,Ly,Lx,4,3)."""
    vals = site_values(name)
    ref = np.array(list(vals.values()))
    got = np.array([field[t, z, y, x, s, c] for (x, y, z, t, s, c) in vals])
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
