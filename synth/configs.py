"""Named synthetic workloads (lattice, gauge-field recipe, right-hand sides, method
parameters).  The paper's ensembles (Tables 1 and 2) are unavailable; these
seeded fields stand in for them at c_sw = 1.0 (the value of Table 2), with the
bare mass m0 chosen near the point where the smallest singular value of D
reaches the stated target (measured by inverse iteration with this library,
``python -m paper_1202_2462_gb300.tune``): 8^4 at m0 = -0.19 has
sigma_min(D) = 1.0e-2.  On these fields sigma_min(D) is close to
0.9 |m0 - m_c| on both sides of a critical mass m_c where the lowest real
eigenvalue of D crosses zero; beyond it (m0 < m_c) D has eigenvalues with
negative real part, the Schwarz smoother no longer damps them and the
multilevel iteration count grows quickly, so "near-critical" is taken on the
physical side m0 > m_c.  32^3 x 64 (eps 0.6): sigma_min = 0.11 at m0 = -0.6,
0.064 at -0.8, 0.081 / 0.098 / 0.115 / 0.133 at -0.82 / -0.84 / -0.86 / -0.88,
7.4e-3 at -0.715, hence m_c = -0.723; the workload uses m0 = -0.7197 with
sigma_min = 3.3e-3 (the near-critical target of 3e-3).
16^3 x 32 (eps 0.5): sigma_min = 0.096 / 0.0026 / 0.042 / 0.088 / 0.133 / 0.178
at m0 = -0.40 / -0.50 / -0.55 / -0.60 / -0.65 / -0.70.

``m0`` is the bare mass in D = 4 + m0 - (hopping)/2 + clover; it maps to the
hopping parameter as m0 = 1/(2 kappa) - 4.

The 32^3 x 64 method parameters (20 set-up sweeps, n_MR = 5, one
post-smoothing sweep, 20 coarse GMRES steps, N = 20, FGMRES(14)) are the
fastest of five scans of these parameters at m0 = -0.7197 (time to solution
of the 12 point sources; the set-up time is reported separately).

``fp64_iterations_per_rhs`` scales the reference arm's timed oracle iteration
to a whole solve: the outer iterations per right-hand side of the method's
plain FP64 form on that workload, as the library's FP64 form reports them
(the FP64 form computes the oracle's iteration: its cycle matches the
oracle's to 1e-11); None where no full-size FP64 solve was run (the reference
arm then reports itself unavailable for that workload).
"""

METRIC = "time-to-solution to 1e-10 at 32^3x64 (mixed vs FP64); Dirac-apply HBM GB/s"

WORKLOADS = {
    # Plain method, FP64, two levels.
    "8^4": dict(
        dims=(8, 8, 8, 8), eps=0.3, gauge_seed=101, c_sw=1.0, m0=-0.19,
        rhs="gaussian", rhs_seed=201, n_levels=2, agg=((4, 4, 4, 4),), n_vec=(8,),
        n_mr=4, nu_post=2, setup_iters=3, coarse_iters=12, fgmres_m=20, tol=1e-10,
        precision="fp64", metric=METRIC, fp64_iterations_per_rhs=None),
    # Plain vs mixed precision, three levels (m0 = -0.50: sigma_min = 2.6e-3,
    # measured with two levels; the three-level form has not been run at it).
    "16^3x32": dict(
        dims=(16, 16, 16, 32), eps=0.5, gauge_seed=102, c_sw=1.0, m0=-0.50,
        rhs="z2", rhs_seed=202, n_levels=3, agg=((4, 4, 4, 4), (2, 2, 2, 2)), n_vec=(20, 20),
        n_mr=4, nu_post=2, setup_iters=3, coarse_iters=12, fgmres_m=20, tol=1e-10,
        precision="fp16", metric=METRIC, fp64_iterations_per_rhs=None),
    # Multi-RHS: 12 spin-colour point sources.
    "32^3x64": dict(
        dims=(32, 32, 32, 64), eps=0.6, gauge_seed=103, c_sw=1.0, m0=-0.7197,
        rhs="point12", rhs_seed=0, n_levels=2, agg=((4, 4, 4, 4), (2, 2, 2, 2)), n_vec=(20, 20),
        n_mr=5, nu_post=1, setup_iters=20, coarse_iters=20, fgmres_m=14, tol=1e-10,
        precision="bf16", metric=METRIC, fp64_iterations_per_rhs=66),
    # Full form at scale: three levels, 24 test vectors proposed by the learned
    # set-up (trained on 16^4 fields of this eps at this m0) and refined by the
    # bootstrap; the 12 point sources in batches of two with FGMRES(12) (the
    # flexible basis of 12 systems in lockstep would not fit beside the
    # hierarchy).  m0 from paper_1202_2462_gb300.tune.find_m0: sigma_min =
    # 9.3e-4 by inverse iteration (critical mass of this field about -0.9762).
    "48^3x96": dict(
        dims=(48, 48, 48, 96), eps=0.7, gauge_seed=105, c_sw=1.0, m0=-0.9752,
        rhs="point12", rhs_seed=0, n_levels=3, agg=((4, 4, 4, 4), (2, 2, 2, 2)), n_vec=(24, 24),
        n_mr=5, nu_post=1, setup_iters=20, coarse_iters=20, fgmres_m=12, tol=1e-10, maxiter=2000,
        inner_iters=4, nrhs_max=2, init="learned", precision="bf16", metric=METRIC, fp64_iterations_per_rhs=None),
    # Mid-size case for Nsight Compute captures: fields larger than L2, a few GB on the device.
    "32^3x32": dict(
        dims=(32, 32, 32, 32), eps=0.6, gauge_seed=104, c_sw=1.0, m0=-0.8,
        rhs="gaussian", rhs_seed=204, n_levels=2, agg=((4, 4, 4, 4),), n_vec=(12,),
        n_mr=4, nu_post=2, setup_iters=2, coarse_iters=12, fgmres_m=10, tol=1e-10, maxiter=30,
        precision="bf16", metric=METRIC, fp64_iterations_per_rhs=None),
    # 12 point sources on the 16^3 x 32 field with the 32^3 x 64 method parameters:
    # the multilevel-vs-CGN comparison across bare masses (bench.py --cgn --m0 ...).
    "16^3x32-12rhs-solve": dict(
        dims=(16, 16, 16, 32), eps=0.5, gauge_seed=102, c_sw=1.0, m0=-0.55,
        rhs="point12", rhs_seed=0, n_levels=2, agg=((4, 4, 4, 4), (2, 2, 2, 2)), n_vec=(20, 20),
        n_mr=4, nu_post=1, setup_iters=8, coarse_iters=16, fgmres_m=20, tol=1e-10, maxiter=2000,
        precision="bf16", metric=METRIC, fp64_iterations_per_rhs=None),
    # 12 point sources on a small lattice: Nsight Compute captures of the multi-RHS kernels.
    "16^3x32-12rhs": dict(
        dims=(16, 16, 16, 32), eps=0.5, gauge_seed=102, c_sw=1.0, m0=-0.55,
        rhs="point12", rhs_seed=0, n_levels=2, agg=((4, 4, 4, 4),), n_vec=(20,),
        n_mr=4, nu_post=2, setup_iters=2, coarse_iters=12, fgmres_m=6, tol=1e-10, maxiter=12,
        precision="bf16", metric=METRIC, fp64_iterations_per_rhs=None),
}


def workload(name):
    """A copy of the named workload's parameter dict."""
    return dict(WORKLOADS[name])
