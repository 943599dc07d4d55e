"""Checkpoint and resume of a set-up (mg_save, mg_setup_load): the set-up of
Sec. 3 is built once and serves every later solve, so its test vectors can be
written to a file and a later context built from them without the bootstrap.
The reloaded context must have the same coarse operators and give the same
solves; a file that does not match the parameters, or is damaged, is
rejected."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from tests.gpu_util import torch_cuda, dev, host, rel

pytestmark = pytest.mark.gpu

CSW = 1.0


def _coarse(torch, G, s, level, nsites, n2):
    m = torch.empty((nsites, 9, n2, n2), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, level, m)
    return host(m)


@pytest.mark.parametrize("levels", [2, 3])
def test_saved_setup_reproduces_the_hierarchy(levels, tmp_path):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    if levels == 2:
        dims, m0, kw = (8, 8, 8, 8), -0.2, dict(n_levels=2, n_vec=(6,))
        sites = [(1, 16, 12)]
    else:
        dims, m0 = (16, 8, 8, 16), -0.1
        kw = dict(n_levels=3, n_vec=(6, 4), sap_block2=(2, 1, 1, 2), agg2=(2, 2, 2, 2), inner_iters=3)
        sites = [(1, 64, 12), (2, 4, 8)]
    u = synth.random_gauge_field(dims, 0.4, 151)
    b = dev(torch, synth.random_spinor(dims, 152))
    path = str(tmp_path / "setup.bin")
    s = G.Solver(dev(torch, u), CSW, m0, setup_iters=2, setup2_iters=1, precision="fp64", seed=3, **kw)
    s.save(path)
    z0, i0, c0 = s.solve(b)
    ref = [_coarse(torch, G, s, lv, ns, n2) for lv, ns, n2 in sites]
    s.close()
    t = G.Solver(dev(torch, u), CSW, m0, precision="fp64", load=path, **kw)
    got = [_coarse(torch, G, t, lv, ns, n2) for lv, ns, n2 in sites]
    z1, i1, c1 = t.solve(b)
    t.close()
    for g, r in zip(got, ref):
        assert np.max(np.abs(g - r)) < 1e-13 * np.max(np.abs(r))
    assert c0 == c1 == 0 and abs(i0.iterations - i1.iterations) <= 1
    assert rel(host(z1), host(z0)) < 1e-8
    # the saved FP64 vectors also serve a mixed-precision context
    op = WilsonClover(u, m0, CSW)
    t = G.Solver(dev(torch, u), CSW, m0, precision="bf16", load=path, **kw)
    z2, i2, c2 = t.solve(b)
    t.close()
    assert c2 == 0
    assert np.linalg.norm(host(b) - op.apply(host(z2))) <= 1e-10 * np.linalg.norm(host(b))


def test_load_rejects_mismatches_and_damage(tmp_path):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims, m0 = (8, 8, 8, 8), -0.2
    u = dev(torch, synth.random_gauge_field(dims, 0.4, 153))
    path = tmp_path / "setup.bin"
    s = G.Solver(u, CSW, m0, n_levels=2, n_vec=(6,), setup_iters=1, precision="fp64")
    s.save(str(path))
    s.close()
    data = path.read_bytes()
    bad = tmp_path / "bad.bin"
    bad.write_bytes(data[:200] + bytes([data[200] ^ 0x40]) + data[201:])     # a byte of the vectors
    short = tmp_path / "short.bin"
    short.write_bytes(data[:len(data) // 2])
    cases = [(str(path), m0, dict(n_vec=(8,)), "differ"), (str(path), -0.25, {}, "m0"),
             (str(bad), m0, {}, "checksum"), (str(short), m0, {}, "truncated"),
             (str(tmp_path / "missing.bin"), m0, {}, "cannot open")]
    for p, mm, extra, word in cases:
        with pytest.raises(G.MgError) as e:
            G.Solver(u, CSW, mm, load=p, **dict(dict(n_levels=2, n_vec=(6,), precision="fp64"), **extra))
        assert e.value.code == G.MG_ERR_ARG and word in str(e.value), (p, str(e.value))
