"""Bare-mass tuning: the smallest singular value of D by inverse iteration.

sigma_min(D)^2 is the smallest eigenvalue of D^dagger D.  Because D is
gamma_5-Hermitian (D^dagger = gamma_5 D gamma_5), (D^dagger D)^{-1} x =
D^{-1} gamma_5 D^{-1} gamma_5 x, so every inverse-iteration step costs two
solves with the library's own solver.  The estimate after each step is
sqrt(<x, x> / <x, (D^dagger D)^{-1} x>) for the normalised iterate x.

Usage (GPU):  python -m paper_1202_2462_gb300.tune --workload 8^4 --m0 -0.2 -0.25
"""

import argparse
import json
import os
import sys

import torch


def gamma5(x):
    y = x.clone()
    y[..., 2:, :] *= -1.0
    return y


def sigma_min(solver, shape, iters=12, seed=0):
    """Inverse-iteration estimate of sigma_min(D) with a Solver (returns the history)."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)
    x = x / torch.linalg.vector_norm(x)
    hist = []
    for _ in range(iters):
        y, _, _ = solver.solve(gamma5(x))
        y, _, _ = solver.solve(gamma5(y))
        lam = torch.vdot(x.flatten(), y.flatten()).real.item()     # <x, (D^dag D)^{-1} x>
        hist.append(1.0 / lam ** 0.5)
        x = y / torch.linalg.vector_norm(y)
    return hist


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import synth
    from paper_1202_2462_gb300 import Solver

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="8^4")
    ap.add_argument("--m0", type=float, nargs="+", required=True)
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--levels", type=int, default=2)
    a = ap.parse_args()
    wl = synth.workload(a.workload)
    u = torch.from_numpy(synth.random_gauge_field(wl["dims"], wl["eps"], wl["gauge_seed"])).cuda()
    shape = u.shape[:4] + (4, 3)
    for m0 in a.m0:
        s = Solver(u, wl["c_sw"], m0, n_levels=a.levels, n_vec=(wl["n_vec"][0],), precision="fp32",
                   tol=1e-9, maxiter=4000, seed=5)
        h = sigma_min(s, shape, a.iters)
        s.close()
        print(json.dumps({"workload": a.workload, "m0": m0, "sigma_min": h[-1], "history": h}), flush=True)


if __name__ == "__main__":
    main()
