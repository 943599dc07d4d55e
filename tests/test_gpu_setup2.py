"""GPU parity of the set-up's second part (Sec. 3: harmonic Ritz pairs of D_c,
S(lambda) smoothing, the (DV)^dagger DV reduction) against the oracle,
through mg_setup with setup2_iters > 0."""

import numpy as np
import pytest

import synth
from oracle import setup2
from oracle.aggregation import Aggregation
from oracle.dirac import WilsonClover
from oracle.mg import Multigrid
from tests.gpu_util import torch_cuda, dev, host, rel

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
M0, CSW = -0.2, 1.0
N = 6


@pytest.fixture(scope="module")
def field():
    u = synth.random_gauge_field(DIMS, 0.4, 31)
    return u, WilsonClover(u, M0, CSW)


def _start():
    rng = np.random.default_rng(1)
    return rng.normal(size=(2, 2, 2, 2, 2 * N)) + 1j * rng.normal(size=(2, 2, 2, 2, 2 * N))


def _oracle(op, iv, part2):
    mg = Multigrid(op, dict(n_levels=2, sap_block=((4, 4, 4, 4),), agg=((4, 4, 4, 4),), n_vec=(N,), setup_iters=1,
                            n_mr=4), init_vectors=iv)
    if part2:
        setup2.part2(mg, 1, _start())
    return mg.levels[0].agg


def test_part2_interpolation_spans_match_the_oracle(field):
    """Same initial vectors and Arnoldi start vector, FP64: the span of the
    local test vectors on every aggregate (the projector P P^dagger, applied to
    random fields) equals the oracle's after part 2, and differs from the
    part-1 span (the comparison is not vacuous)."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, op = field
    iv = synth.test_vector_draw(DIMS, N, 41)
    s = G.Solver(dev(torch, u), CSW, M0, n_levels=2, n_vec=(N,), setup_iters=1, setup2_iters=1, n_mr=4,
                 precision="fp64", init_vectors=dev(torch, iv), setup2_start=dev(torch, _start().reshape(16, 2 * N)))
    v = torch.zeros((N,) + s.lat + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 0, v)
    s.close()
    gpu = Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(host(v))
    ref = _oracle(op, iv, True)
    before = _oracle(op, iv, False)
    for x in synth.random_spinor(DIMS, 77, nvec=3):
        pg = gpu.prolong(gpu.restrict(x))
        pr = ref.prolong(ref.restrict(x))
        assert rel(pg, pr) < 1e-8
        assert rel(before.prolong(before.restrict(x)), pr) > 1e-3


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_hierarchy_with_part2_solves_to_the_tolerance(field, prec):
    """Part 2 with the drawn start vector, plain and mixed form: the solve
    reaches ||b - D z|| <= 1e-10 ||b|| under the oracle's D."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, op = field
    b = synth.random_spinor(DIMS, 78)
    its = {}
    for it2 in (0, 1):
        s = G.Solver(dev(torch, u), CSW, M0, n_levels=2, n_vec=(8,), setup_iters=2, setup2_iters=it2,
                     precision=prec, seed=5)
        z, info, code = s.solve(dev(torch, b))
        s.close()
        assert code == 0
        assert np.linalg.norm(b - op.apply(host(z))) <= 1e-10 * np.linalg.norm(b)
        its[it2] = info.iterations
    print("outer iterations without / with set-up part 2:", its)


def test_part2_three_levels_matches_the_oracle():
    """Three levels (the paper ran two; reading: the harmonic Ritz pairs of the
    coarsest operator are interpolated through level 1 to the fine level,
    smoothed and reduced there, and level 1 is rebuilt from the new vectors as
    part 1 builds it).  Same initial vectors and start vector, FP64: the span
    of the fine-level test vectors on every aggregate and the span of the
    composite interpolation P0 P1 (both invariant to the phases of individual
    vectors) equal the oracle's."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = (16, 8, 8, 16)
    n0, n1, sap2, agg2 = 6, 4, (2, 1, 1, 2), (2, 2, 2, 2)
    u = synth.random_gauge_field(dims, 0.4, 61)
    op = WilsonClover(u, -0.1, CSW)
    iv = synth.test_vector_draw(dims, n0, 62)
    rng = np.random.default_rng(3)
    start = rng.normal(size=(2, 1, 1, 2, 2 * n1)) + 1j * rng.normal(size=(2, 1, 1, 2, 2 * n1))
    s = G.Solver(dev(torch, u), CSW, -0.1, n_levels=3, n_vec=(n0, n1), setup_iters=1, setup2_iters=1, n_mr=4,
                 inner_iters=3, sap_block2=sap2, agg2=agg2, precision="fp64", init_vectors=dev(torch, iv),
                 setup2_start=dev(torch, start.reshape(4, 2 * n1)))
    v0 = torch.zeros((n0,) + s.lat + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 0, v0)
    v1 = torch.zeros((n1, 4, 2, 2, 4, 2 * n0), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 1, v1)
    b = dev(torch, synth.random_spinor(dims, 63))
    z, info, code = s.solve(b)
    s.close()
    assert code == 0 and np.linalg.norm(host(b) - op.apply(host(z))) <= 1e-10 * np.linalg.norm(host(b))
    mg = Multigrid(op, dict(n_levels=3, sap_block=((4, 4, 4, 4), sap2), agg=((4, 4, 4, 4), agg2), n_vec=(n0, n1),
                            setup_iters=1, n_mr=4, inner_iters=3), iv)
    before = Multigrid(op, dict(n_levels=3, sap_block=((4, 4, 4, 4), sap2), agg=((4, 4, 4, 4), agg2),
                                n_vec=(n0, n1), setup_iters=1, n_mr=4, inner_iters=3), iv)
    setup2.part2(mg, 1, start)
    g0 = Aggregation(dims, (4, 4, 4, 4), (4, 3)).build(host(v0))
    g1 = Aggregation(g0.cdims, agg2, (2 * n0,)).build(host(v1))
    r0, r1 = mg.levels[0].agg, mg.levels[1].agg
    b0, b1 = before.levels[0].agg, before.levels[1].agg
    for x in synth.random_spinor(dims, 64, nvec=3):
        assert rel(g0.prolong(g0.restrict(x)), r0.prolong(r0.restrict(x))) < 1e-8
        pg = g0.prolong(g1.prolong(g1.restrict(g0.restrict(x))))
        pr = r0.prolong(r1.prolong(r1.restrict(r0.restrict(x))))
        assert rel(pg, pr) < 1e-7
        assert rel(b0.prolong(b1.prolong(b1.restrict(b0.restrict(x)))), pr) > 1e-3
