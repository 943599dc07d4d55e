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
