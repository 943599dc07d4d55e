"""Parity at the benchmark's full size (32^3 x 64 lattice, 12 right-hand sides,
BF16-stored links and clover, FP32 arithmetic -- the launch configuration of
the timed solve) on sampled outputs the oracle evaluates one by one: the Dirac
operator at sampled sites (Sec. 1, Eq. 1.1) and one red-black Schwarz sweep on
sampled colour-0 blocks (Sec. 2, Algorithm 1), including blocks and sites on
the lattice boundary.  The oracle uses the identically rounded links and
clover, so the tolerance is that of FP32 arithmetic."""

import numpy as np
import pytest

import synth
from oracle.dirac import apply_at_sites
from oracle.sap import colour_pass_on_block
from tests.gpu_util import torch_cuda, host, round_storage

pytestmark = pytest.mark.gpu

W = synth.workload("32^3x64")
NRHS = 12


def _bf16(x):
    return round_storage(x, "bf16")


@pytest.fixture(scope="module")
def big():
    torch = torch_cuda()
    dims = W["dims"]
    u = synth.random_gauge_field(dims, W["eps"], W["gauge_seed"])
    phi = synth.uniform_spinor(dims, 701, 2, synth.rng.STREAM_SPINOR)
    coef = [(1.0 + 0.25 * r) * np.exp(0.4j * r) for r in range(NRHS)]
    # twelve distinct right-hand sides built from two base fields (cheap to draw at this size)
    fields = np.stack([coef[r] * phi[0] + (0.5 - 0.1 * r) * phi[1] for r in range(NRHS)]).astype(np.complex64)
    yield torch, dims, u, fields
    del fields


def test_fullsize_dirac_sampled_sites(big):
    torch, dims, u, psi = big
    import paper_1202_2462_gb300 as G
    s = G.Solver(torch.from_numpy(u).cuda(), W["c_sw"], W["m0"], n_levels=1, precision="bf16", nrhs_max=NRHS,
                 fgmres_m=1)
    out = s.dirac(torch.from_numpy(psi).cuda(), G.MG_BF16)
    torch.cuda.synchronize()
    s.close()
    rng = np.random.default_rng(11)
    lx, ly, lz, lt = dims
    sites = [(0, 0, 0, 0), (lx - 1, ly - 1, lz - 1, lt - 1), (3, 4, 31, 63)] + \
            [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(9)]
    for r in (0, 5, 11):
        ref = apply_at_sites(u, psi[r].astype(np.complex128), W["m0"], W["c_sw"], sites, round_fields=_bf16)
        idx = torch.tensor([((t * lz + z) * ly + y) * lx + x for (x, y, z, t) in sites], device="cuda")
        got = host(out[r].reshape(-1, 4, 3)[idx]).astype(np.complex128)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < 2e-6, (r, err)


def test_fullsize_schwarz_sweep_sampled_blocks(big):
    torch, dims, u, b = big
    import paper_1202_2462_gb300 as G
    z0 = np.ascontiguousarray(b[::-1] * 0.3).astype(np.complex64)     # a different, nonzero start
    s = G.Solver(torch.from_numpy(u).cuda(), W["c_sw"], W["m0"], n_levels=1, precision="bf16", nrhs_max=NRHS,
                 n_mr=W["n_mr"], fgmres_m=1)
    z = torch.from_numpy(z0).cuda()
    s.smooth(torch.from_numpy(b).cuda(), z, 1)
    torch.cuda.synchronize()
    s.close()
    lx, ly, lz, lt = dims
    blocks = [(0, 0, 0, 0), (lx - 4, ly - 4, lz - 4, lt - 4), (4, 4, 0, 0), (8, 12, 20, 40)]
    for o in blocks:
        assert (sum(c // 4 for c in o)) % 2 == 0                       # colour 0: final after the sweep
    for r in (0, 7):
        for (x, y, zz, t) in blocks:
            ref = colour_pass_on_block(u, W["m0"], W["c_sw"], b[r].astype(np.complex128),
                                       z0[r].astype(np.complex128), (x, y, zz, t), W["n_mr"], round_fields=_bf16)
            got = host(z[r, t:t + 4, zz:zz + 4, y:y + 4, x:x + 4]).astype(np.complex128)
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < 5e-6, (r, (x, y, zz, t), err)
