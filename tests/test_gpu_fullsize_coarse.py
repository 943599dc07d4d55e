"""Parity of the coarse-grid side at the benchmark's full size and launch
configuration (32^3 x 64 lattice, N = 20 test vectors so 2N = 40 coarse dof,
12 right-hand sides, BF16 links and clover, FP16-stored P and D_c, FP32
vectors) on sampled aggregates and coarse sites, including the first and last
aggregate and coarse sites that the tensor-core stencil's CTAs reach after
walking several sites (8192 coarse sites on 1216 CTAs: sites 1216 apart share
a CTA, sites from 7296 on are in the last stride).

* Galerkin operator (Sec. 3, Eq. 3.2): at a sampled coarse site a, the oracle
  builds D_c on a 12^4 periodic patch centred on aggregate a from the exact
  links and the library's exported FP64 test vectors (P is an input here; its
  own parity is checked at small size) and compares its nine 40 x 40 blocks
  at the centre with the library's FP64 D_c.  The centre aggregate's
  couplings involve only links, clover and vectors inside the patch's
  interior, so the patch wrap does not reach them.  The mixed form
  assembles D_c in FP32 arithmetic (it stores and applies it in FP32 and
  FP16), so the entries agree to FP32 accuracy, 5e-6 of the largest.
* Restriction P^dagger and interpolation P (Sec. 3) of 12 FP32 vectors at
  once (the cycle's batched tensor-core transfers, TF32 inputs): against the
  oracle's transfers with the FP16-rounded P and TF32-rounded vectors on the
  sampled aggregates.
* D_c x for 12 right-hand sides (the FP16 tensor-core stencil): against
  sum_d M_d(a) x(a + offset_d) with the FP16-rounded operator and vectors.
Element-wise maximum errors relative to the largest reference entry."""

import numpy as np
import pytest

import synth
from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.dirac import WilsonClover, patch
from tests.gpu_util import torch_cuda, host, round_storage

pytestmark = pytest.mark.gpu

W = synth.workload("32^3x64")
NRHS, N = 12, 20
N2 = 2 * N


def _tf32(x):
    """float32 values rounded to TF32 (10-bit mantissa, to nearest, ties away
    from zero), as the tensor-core transfers round their inputs."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32)
    b = ((b.astype(np.uint64) + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _tf32c(z):
    return _tf32(np.real(z)) + 1j * _tf32(np.imag(z))


def _maxrel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def big():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = W["dims"]
    u = synth.random_gauge_field(dims, W["eps"], W["gauge_seed"])
    s = G.Solver(torch.from_numpy(u).cuda(), W["c_sw"], W["m0"], n_levels=2, n_vec=(N,), setup_iters=1,
                 precision="bf16", nrhs_max=NRHS, n_mr=W["n_mr"], coarse_iters=W["coarse_iters"], seed=3)
    lt, lz, ly, lx = u.shape[:4]
    v = torch.empty((N, lt, lz, ly, lx, 4, 3), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 0, v)
    clat = (lt // 4, lz // 4, ly // 4, lx // 4)
    nc = int(np.prod(clat))
    m = torch.empty((nc, 9, N2, N2), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, 1, m)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    sites = sorted({0, 1, 1215, 1216, 2431, 7295, 7296, nc - 1} | {int(k) for k in rng.integers(0, nc, 3)})
    yield torch, G, s, u, v, m, clat, sites
    s.close()


def _coords(a, clat):
    ct, cz, cy, cx = np.unravel_index(a, clat)
    return int(cx), int(cy), int(cz), int(ct)                  # (x, y, z, t)


def _index(coords, clat):
    cx, cy, cz, ct = coords
    return ((ct * clat[1] + cz) * clat[2] + cy) * clat[3] + cx


def _block(torch, f, origin, size):
    """f[..., t, z, y, x, 4, 3] on the periodic box of edge `size` at origin (x, y, z, t), to host."""
    lead = f.dim() - 6
    idx = []
    for mu, o in zip((3, 2, 1, 0), (origin[3], origin[2], origin[1], origin[0])):
        n = f.shape[lead + (3 - mu)]
        idx.append(torch.tensor([(o + k) % n for k in range(size)], device=f.device))
    g = f
    for ax, ix in enumerate(idx):
        g = torch.index_select(g, lead + ax, ix)
    return host(g)


def test_fullsize_coarse_operator_sampled_sites(big):
    torch, G, s, u, v, m, clat, sites = big
    for a in sites:
        c = _coords(a, clat)
        origin = tuple(4 * k - 4 for k in c)
        up = patch(u, origin, 12)
        vp = _block(torch, v, origin, 12)
        agg = Aggregation((12, 12, 12, 12), (4, 4, 4, 4), (4, 3)).build(vp)
        op = CoarseOperator(WilsonClover(up, W["m0"], W["c_sw"]), agg)
        ref = [op.self_[1, 1, 1, 1]]
        for mu in range(4):
            ref += [op.fwd[mu][1, 1, 1, 1], op.bwd[mu][1, 1, 1, 1]]
        ref = np.stack(ref)
        got = host(m[a])
        assert _maxrel(got, ref) < 5e-6, (a, _maxrel(got, ref))


def _rhs(dims, seed):
    phi = synth.uniform_spinor(dims, seed, 2, synth.rng.STREAM_SPINOR)
    coef = [(1.0 + 0.25 * r) * np.exp(0.4j * r) for r in range(NRHS)]
    return np.stack([coef[r] * phi[0] + (0.5 - 0.1 * r) * phi[1] for r in range(NRHS)]).astype(np.complex64)


def test_fullsize_restrict_prolong_sampled_aggregates(big):
    torch, G, s, u, v, m, clat, sites = big
    dims = W["dims"]
    nc = int(np.prod(clat))
    r = torch.from_numpy(_rhs(dims, 711)).cuda()
    rc = torch.zeros((NRHS, nc, N2), dtype=torch.complex64, device="cuda")
    G.mg_restrict_batch(s.ctx, 0, r, rc, G.MG_BF16, NRHS)
    e = synth.uniform_spinor((8, 8, 8, 16), 712, NRHS, synth.rng.STREAM_SPINOR)      # 8192 coarse sites x 12
    e = np.concatenate([e.reshape(NRHS, nc, 12)] * 4, axis=-1)[..., :N2]
    e = (e * np.linspace(0.5, 1.5, N2)).astype(np.complex64)
    ed = torch.from_numpy(np.ascontiguousarray(e)).cuda()
    f = torch.zeros_like(r)
    G.mg_prolong_batch(s.ctx, 0, ed, f, G.MG_BF16, NRHS)
    torch.cuda.synchronize()
    for a in sites:
        c = _coords(a, clat)
        origin = tuple(4 * k for k in c)
        agg = Aggregation((4, 4, 4, 4), (4, 4, 4, 4), (4, 3)).build(_block(torch, v, origin, 4))
        agg.q = round_storage(agg.q, "fp16")
        ref = agg.restrict(_tf32c(_block(torch, r, origin, 4))).reshape(NRHS, N2)
        got = host(rc[:, a]).astype(np.complex128)
        assert _maxrel(got, ref) < 1e-5, ("restrict", a, _maxrel(got, ref))
        ref = agg.prolong(_tf32c(e[:, a]).reshape(NRHS, 1, 1, 1, 1, N2))
        got = _block(torch, f, origin, 4).astype(np.complex128)
        assert _maxrel(got, ref) < 1e-5, ("prolong", a, _maxrel(got, ref))


def test_fullsize_coarse_stencil_sampled_sites(big):
    torch, G, s, u, v, m, clat, sites = big
    nc = int(np.prod(clat))
    x = synth.uniform_spinor((8, 8, 8, 16), 713, NRHS, synth.rng.STREAM_SPINOR).reshape(NRHS, nc, 12)
    x = np.concatenate([x, 0.5 * x, -x, x[..., :4]], axis=-1).astype(np.complex64)   # 40 dof
    out = torch.zeros((NRHS, nc, N2), dtype=torch.complex64, device="cuda")
    G.mg_coarse_apply_batch(s.ctx, 1, torch.from_numpy(np.ascontiguousarray(x)).cuda(), out, G.MG_FP32, NRHS)
    torch.cuda.synchronize()
    x16 = round_storage(x.astype(np.complex128), "fp16")
    for a in sites:
        c = _coords(a, clat)
        ma = round_storage(host(m[a]), "fp16")
        ref = ma[0] @ x16[:, a].T
        for mu in range(4):
            for d, step in ((1 + 2 * mu, 1), (2 + 2 * mu, -1)):
                cn = list(c)
                n = clat[3 - mu]
                cn[mu] = (cn[mu] + step) % n
                ref = ref + ma[d] @ x16[:, _index(cn, clat)].T
        got = host(out[:, a]).astype(np.complex128)
        assert _maxrel(got, ref.T) < 5e-6, (a, _maxrel(got, ref.T))
