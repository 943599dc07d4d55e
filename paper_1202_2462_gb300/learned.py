"""Learned set-up: a gauge-covariant convolutional network that proposes
near-kernel test vectors from noise.  It is trained to imitate the bootstrap
set-up's smoothing (nu Schwarz sweeps of the smoother's iteration matrix on
D x = 0 started at the noise, Sec. 3); the plain bootstrap stays the fallback
and refines whatever the network proposes.

Every step runs in the library's kernels: the transport layers, the gate,
the loss and the Adam update (mg_net_*, mg_adam_step); this module only
keeps the weights and activations (device tensors) and sequences the calls.
Fields are complex64 tensors in the library's blocked layout (mg_pack_spinor),
one channel per 12V complex numbers.
"""

import math

import torch

from . import binding as B


class GaugeNet:
    """Layers (cin -> cout): 1 -> C -> ... -> C -> 1, gates between layers."""

    def __init__(self, channels=16, layers=3, seed=0):
        if layers < 2:
            raise ValueError("at least two layers")
        self.shapes = [(channels, 1)] + [(channels, channels)] * (layers - 2) + [(1, channels)]
        gen = torch.Generator().manual_seed(seed)
        self.weights = []
        for cout, cin in self.shapes:
            std = 1.0 / math.sqrt(cin * 9 * 4 * 2)
            w = torch.randn((cout, cin, 9, 4, 4, 2), generator=gen, dtype=torch.float32) * std
            self.weights.append(torch.view_as_complex(w).cuda().contiguous())
        self.m = [torch.zeros_like(torch.view_as_real(w)) for w in self.weights]
        self.v = [torch.zeros_like(torch.view_as_real(w)) for w in self.weights]
        self.steps = 0

    # ------------------------------------------------------------------ passes
    def forward(self, s, eta):
        """Network output for the blocked noise field eta; returns (out, cache)."""
        fs = eta.numel()
        x = eta
        cache = []
        last = len(self.shapes) - 1
        for i, ((cout, cin), w) in enumerate(zip(self.shapes, self.weights)):
            y = torch.empty(cout * fs, dtype=torch.complex64, device="cuda")
            B.mg_net_layer_forward(s.ctx, cin, cout, w, x, y)
            cache.append((x, y))
            if i < last:
                z = torch.empty_like(y)
                B.mg_net_gate_forward(s.ctx, cout, y, z)
                x = z
            else:
                x = y
        return x, cache

    def forward_bf16(self, s, eta):
        """Inference with BF16 storage: the weights rounded to BF16 and the
        context's BF16 links (a BF16 context), FP32 activations."""
        fs = eta.numel()
        x = eta
        last = len(self.shapes) - 1
        for i, ((cout, cin), w) in enumerate(zip(self.shapes, self.weights)):
            wb = torch.view_as_real(w).to(torch.bfloat16).contiguous()
            y = torch.empty(cout * fs, dtype=torch.complex64, device="cuda")
            B.mg_net_layer_forward_bf16(s.ctx, cin, cout, wb, x, y)
            if i < last:
                z = torch.empty_like(y)
                B.mg_net_gate_forward(s.ctx, cout, y, z)
                x = z
            else:
                x = y
        return x

    def backward(self, s, out, cache, target):
        """Loss ||out - target||^2 / ||target||^2 and the weight gradients."""
        g = torch.empty_like(out)
        loss = B.mg_net_loss(s.ctx, out, target, g)
        grads = [None] * len(self.weights)
        last = len(self.shapes) - 1
        for i in range(last, -1, -1):
            cout, cin = self.shapes[i]
            x, y = cache[i]
            if i < last:
                gg = torch.empty_like(y)
                B.mg_net_gate_backward(s.ctx, cout, y, g, gg)
                g = gg
            gw = torch.empty_like(self.weights[i])
            gx = torch.empty_like(x) if i > 0 else None
            B.mg_net_layer_backward(s.ctx, cin, cout, self.weights[i], x, g, gx, gw)
            grads[i] = gw
            g = gx
        return loss, grads

    def adam(self, s, grads, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
        self.steps += 1
        for w, g, m, v in zip(self.weights, grads, self.m, self.v):
            p = torch.view_as_real(w)
            B.mg_adam_step(s.ctx, p.numel(), p, torch.view_as_real(g), m, v, lr, beta1, beta2, eps, self.steps)

    # ------------------------------------------------------------------ data
    @staticmethod
    def blocked(s, canonical):
        """Canonical complex64 field(s) -> blocked layout."""
        n = 1 if canonical.dim() == 6 else canonical.shape[0]
        out = torch.empty(canonical.numel(), dtype=torch.complex64, device="cuda")
        B.mg_pack_spinor(s.ctx, canonical.contiguous(), out, B.MG_FP32, n)
        return out

    @staticmethod
    def canonical(s, blocked, nrhs=1):
        out = torch.empty((nrhs,) + s.lat + (4, 3), dtype=torch.complex64, device="cuda")
        B.mg_unpack_spinor(s.ctx, blocked, out, B.MG_FP32, nrhs)
        return out

    @staticmethod
    def smoothed(s, eta_canonical, sweeps):
        """The bootstrap's smoothing of eta: `sweeps` Schwarz sweeps on D x = 0
        from x = eta (the smoother's iteration matrix applied), rescaled to
        eta's norm (the set-up keeps only directions)."""
        z = eta_canonical.clone()
        b = torch.zeros_like(z)
        s.smooth(b, z, sweeps)
        return z * (torch.linalg.vector_norm(eta_canonical) / torch.linalg.vector_norm(z))

    def propose(self, s, eta_canonical, bf16=False):
        """Network output for canonical noise fields (N, ...) as canonical
        complex64; bf16: BF16 inference (s a BF16 context)."""
        outs = []
        for k in range(eta_canonical.shape[0]):
            x = self.blocked(s, eta_canonical[k])
            out = self.forward_bf16(s, x) if bf16 else self.forward(s, x)[0]
            outs.append(self.canonical(s, out)[0])
        return torch.stack(outs)


def train(c_sw, m0, train_dims=(16, 16, 16, 16), train_fields=20, eps_train=0.5, sweeps=2, channels=16,
          layers=3, epochs=4, lr=1e-2, seed=1000):
    """Train a GaugeNet on seeded fields U = exp(i eps_train H) of train_dims
    (four noise fields each, `epochs` passes): input noise, target the
    bootstrap-smoothed noise at (c_sw, m0).  Returns (net, losses, seconds of
    training on the device)."""
    import time
    import synth
    from .solver import Solver
    net = GaugeNet(channels=channels, layers=layers, seed=seed)
    losses = []
    t_train = 0.0
    for f in range(train_fields):
        u = torch.from_numpy(synth.random_gauge_field(train_dims, eps_train, seed + f)).cuda()
        s = Solver(u, c_sw, m0, n_levels=1, precision="fp32", fgmres_m=2)
        eta = torch.from_numpy(synth.random_spinor(train_dims, seed + 100 + f, nvec=4)).to(torch.complex64).cuda()
        inputs = [GaugeNet.blocked(s, eta[k]) for k in range(4)]
        targets = [GaugeNet.blocked(s, GaugeNet.smoothed(s, eta[k], sweeps)) for k in range(4)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ep in range(epochs):
            for k in range(4):
                out, cache = net.forward(s, inputs[k])
                val, grads = net.backward(s, out, cache, targets[k])
                net.adam(s, grads, lr=lr)
                losses.append(val)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        s.close()
    return net, losses, t_train


def infer(net, u, c_sw, m0, noise):
    """BF16 inference of the network's proposals for the noise fields (N, ...)
    on the gauge field u (device, canonical); returns (proposals as complex64
    in the canonical layout, which mg_params.init_vectors takes, and seconds).
    One field at a time, written straight into the output.  Raises if a
    proposal is not finite."""
    import time
    from .solver import Solver
    s = Solver(u, c_sw, m0, n_levels=1, precision="bf16", fgmres_m=2)
    out = torch.empty(noise.shape, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(noise.shape[0]):
        out[k] = net.propose(s, noise[k:k + 1].to(torch.complex64), bf16=True)[0]
    torch.cuda.synchronize()
    t_infer = time.perf_counter() - t0
    s.close()
    if not bool(torch.isfinite(torch.view_as_real(out)).all()):
        raise RuntimeError("the network's proposals are not finite")
    return out, t_infer


def study(train_dims=(16, 16, 16, 16), train_fields=20, eps_train=0.5, eval_workload="32^3x64", n_vec=24,
          sweeps=2, channels=16, layers=3, epochs=4, lr=1e-2, setup_iters=(1, 2, 4, 8, 20), seed=1000):
    """Train on seeded fields (noise -> bootstrap-smoothed noise, FP32), propose
    the evaluation lattice's test vectors (BF16 inference), and compare
    hierarchies built from the proposals and from plain noise, each refined by
    the same number of bootstrap sweeps: set-up time (with the inference time
    for the network), outer iterations per right-hand side of the 12
    point-source solve, and the average residual reduction per outer
    iteration rho = relres^(1 / iterations).  Returns a dict; 'equal_time'
    pairs each network row with the noise row whose set-up took at least as
    long."""
    import time
    import synth
    from .solver import Solver
    wl = synth.workload(eval_workload)
    net, losses, t_train = train(wl["c_sw"], wl["m0"], train_dims, train_fields, eps_train, sweeps, channels,
                                 layers, epochs, lr, seed)
    dims = tuple(wl["dims"])
    u = torch.from_numpy(synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"])).cuda()
    noise = torch.from_numpy(synth.test_vector_draw(dims, n_vec, seed + 7)).cuda()
    prop, t_infer = infer(net, u, wl["c_sw"], wl["m0"], noise)
    import numpy as np
    b = torch.from_numpy(np.ascontiguousarray(synth.point_sources(dims))).cuda()
    rows = []
    for k in setup_iters:
        for name, iv in (("noise", noise), ("network", prop)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = Solver(u, wl["c_sw"], wl["m0"], n_levels=2, n_vec=(n_vec,), setup_iters=k, n_mr=wl["n_mr"],
                         nu_post=wl["nu_post"], coarse_iters=wl["coarse_iters"], fgmres_m=wl["fgmres_m"],
                         precision=wl["precision"], nrhs_max=12, init_vectors=iv, maxiter=2000)
            torch.cuda.synchronize()
            ts = time.perf_counter() - t0 + (t_infer if name == "network" else 0.0)
            t0 = time.perf_counter()
            try:
                z, info, code = sol.solve(b)
            except B.MgError as e:                       # recorded, not fatal: the row reports the failure
                sol.close()
                rows.append(dict(init=name, setup_iters=k, setup_s=ts, status=e.code, error=str(e)))
                continue
            torch.cuda.synchronize()
            tsol = time.perf_counter() - t0
            sol.close()
            its = info.iterations / 12
            rows.append(dict(init=name, setup_iters=k, setup_s=ts, solve_s=tsol, iterations_per_rhs=its,
                             rho=float(info.relres ** (1.0 / its)) if its > 0 else None,
                             relres=info.relres, status=code))
    equal = []
    for r in rows:
        if r["init"] != "network" or r["status"] != 0:
            continue
        slower = [q for q in rows if q["init"] == "noise" and q["status"] == 0 and q["setup_s"] >= r["setup_s"]]
        if slower:
            q = min(slower, key=lambda q: q["setup_s"])
            equal.append(dict(network_sweeps=r["setup_iters"], noise_sweeps=q["setup_iters"],
                              network_setup_s=r["setup_s"], noise_setup_s=q["setup_s"],
                              network_its=r["iterations_per_rhs"], noise_its=q["iterations_per_rhs"]))
    return dict(train_loss_first=float(sum(losses[:8]) / 8), train_loss_last=float(sum(losses[-8:]) / 8),
                train_s=t_train, inference_s=t_infer, inference="bf16", n_vec=n_vec, sweeps_imitated=sweeps,
                m0=wl["m0"], rows=rows, equal_time=equal)


if __name__ == "__main__":
    import json
    print(json.dumps(study()))
