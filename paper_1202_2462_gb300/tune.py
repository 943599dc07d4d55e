"""Bare-mass tuning: the smallest singular value of D by inverse iteration.

sigma_min(D)^2 is the smallest eigenvalue of D^dagger D.  Because D is
gamma_5-Hermitian (D^dagger = gamma_5 D gamma_5), (D^dagger D)^{-1} x =
D^{-1} gamma_5 D^{-1} gamma_5 x, so every inverse-iteration step costs two
solves with the library's own solver.  The estimate after each step is
sqrt(<x, x> / <x, (D^dagger D)^{-1} x>) for the normalised iterate x.

Usage (GPU):  python -m paper_1202_2462_gb300.tune --workload 8^4 --m0 -0.2 -0.25
              python -m paper_1202_2462_gb300.tune --workload 48^3x96 --m0 -0.85 --find 1e-3
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


def find_m0(make_solver, shape, m_start, target, slope=0.9, iters=10, max_steps=8, log=None):
    """A bare mass with sigma_min(D) near `target` on the physical side of the
    critical mass m_c (the mass below which D has eigenvalues with negative
    real part).  On these fields sigma_min falls linearly as m0 approaches
    m_c, sigma_min ~ slope * (m0 - m_c), so each step measures sigma_min at
    the current m0 (a fresh solver from make_solver(m0)), takes the slope of
    the last two points (the given slope on the first step), estimates m_c,
    and moves to m_c + max(target, sigma / 3) / slope: at most two thirds of
    the way at once, because the inverse-iteration estimate is an upper bound
    and a step past m_c would leave the physical side.  m_start must lie on
    that side.  Stops once sigma_min is within 25% of target; returns
    (m0, sigma_min, steps) with steps a list of (m0, sigma_min)."""
    pts = []
    m = m_start
    for _ in range(max_steps):
        s = make_solver(m)
        sig = sigma_min(s, shape, iters)[-1]
        s.close()
        if pts and sig >= pts[-1][1]:
            raise RuntimeError(f"sigma_min did not fall from m0 = {pts[-1][0]} to {m}: past the critical mass?")
        pts.append((m, sig))
        if log:
            log({"m0": m, "sigma_min": sig})
        if abs(sig - target) <= 0.25 * target:
            return m, sig, pts
        if len(pts) > 1:
            (m1, s1), (m2, s2) = pts[-2], pts[-1]
            slope = (s1 - s2) / (m1 - m2)
        m_c = m - sig / slope
        m = m_c + max(target, sig / 3.0) / slope
    raise RuntimeError(f"no bare mass with sigma_min within 25% of {target} after {max_steps} steps: {pts}")


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
    ap.add_argument("--find", type=float, default=None,
                    help="search from the first --m0 (physical side) for sigma_min near this value (find_m0)")
    a = ap.parse_args()
    wl = synth.workload(a.workload)
    u = torch.from_numpy(synth.random_gauge_field(wl["dims"], wl["eps"], wl["gauge_seed"])).cuda()
    shape = u.shape[:4] + (4, 3)
    if a.find is not None:
        make = lambda m0: Solver(u, wl["c_sw"], m0, n_levels=2, n_vec=(wl["n_vec"][0],), setup_iters=6,
                                 precision="fp32", tol=1e-9, maxiter=4000, seed=5)
        log = lambda d: print(json.dumps(dict(d, workload=a.workload)), flush=True)
        m0, sig, pts = find_m0(make, shape, a.m0[0], a.find, iters=a.iters, log=log)
        print(json.dumps({"workload": a.workload, "found_m0": m0, "sigma_min": sig, "steps": pts}), flush=True)
        return
    for m0 in a.m0:
        s = Solver(u, wl["c_sw"], m0, n_levels=a.levels, n_vec=(wl["n_vec"][0],), precision="fp32",
                   tol=1e-9, maxiter=4000, seed=5)
        h = sigma_min(s, shape, a.iters)
        s.close()
        print(json.dumps({"workload": a.workload, "m0": m0, "sigma_min": h[-1], "history": h}), flush=True)


if __name__ == "__main__":
    main()
