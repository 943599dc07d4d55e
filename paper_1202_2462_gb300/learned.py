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

    def propose(self, s, eta_canonical):
        """Network output for canonical noise fields (N, ...) as canonical complex64."""
        outs = []
        for k in range(eta_canonical.shape[0]):
            out, _ = self.forward(s, self.blocked(s, eta_canonical[k]))
            outs.append(self.canonical(s, out)[0])
        return torch.stack(outs)


def study(train_dims=(16, 16, 16, 16), train_fields=20, eps_train=0.5, eval_workload="32^3x64", n_vec=24,
          sweeps=2, channels=16, layers=3, epochs=4, lr=1e-2, setup_iters=(2, 8), seed=1000):
    """Train on seeded fields (noise -> bootstrap-smoothed noise), propose the
    evaluation lattice's test vectors, and compare set-up time and outer
    iterations of hierarchies built from the proposals and from plain noise
    with the same number of bootstrap sweeps.  Returns a dict."""
    import time
    import synth
    from .solver import Solver
    wl = synth.workload(eval_workload)
    net = GaugeNet(channels=channels, layers=layers, seed=seed)
    losses = []
    t_train = 0.0
    for f in range(train_fields):
        u = torch.from_numpy(synth.random_gauge_field(train_dims, eps_train, seed + f)).cuda()
        s = Solver(u, wl["c_sw"], wl["m0"], n_levels=1, precision="fp32", fgmres_m=2)
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
    dims = tuple(wl["dims"])
    u = torch.from_numpy(synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"])).cuda()
    noise = torch.from_numpy(synth.test_vector_draw(dims, n_vec, seed + 7)).to(torch.complex64).cuda()
    s = Solver(u, wl["c_sw"], wl["m0"], n_levels=1, precision="fp32", fgmres_m=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prop = net.propose(s, noise)
    torch.cuda.synchronize()
    t_infer = time.perf_counter() - t0
    s.close()
    import numpy as np
    b = torch.from_numpy(np.ascontiguousarray(synth.point_sources(dims))).cuda()
    rows = []
    for k in setup_iters:
        for name, iv in (("noise", noise), ("network", prop)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = Solver(u, wl["c_sw"], wl["m0"], n_levels=2, n_vec=(n_vec,), setup_iters=k, n_mr=wl["n_mr"],
                         nu_post=wl["nu_post"], coarse_iters=wl["coarse_iters"], fgmres_m=wl["fgmres_m"],
                         precision=wl["precision"], nrhs_max=12, init_vectors=iv.to(torch.complex128).contiguous())
            torch.cuda.synchronize()
            ts = time.perf_counter() - t0
            t0 = time.perf_counter()
            z, info, code = sol.solve(b)
            torch.cuda.synchronize()
            tsol = time.perf_counter() - t0
            sol.close()
            rows.append(dict(init=name, setup_iters=k, setup_s=ts, solve_s=tsol, iterations_per_rhs=info.iterations / 12,
                             relres=info.relres, status=code))
    return dict(train_loss_first=float(sum(losses[:8]) / 8), train_loss_last=float(sum(losses[-8:]) / 8),
                train_s=t_train, inference_s=t_infer, n_vec=n_vec, sweeps_imitated=sweeps, rows=rows)


if __name__ == "__main__":
    import json
    print(json.dumps(study()))
