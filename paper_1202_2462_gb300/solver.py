"""Torch convenience wrapper around the C-ABI (marshalling only)."""

import torch

from . import binding as B

_ARRAYS = {"dims": 4, "agg2": 4, "sap_block2": 4, "n_vec": 2}


def make_params(dims, **kw):
    """mg_params with the library defaults, dims and any overrides."""
    p = B.mg_default_params()
    for mu in range(4):
        p.dims[mu] = int(dims[mu])
    for key, val in kw.items():
        if key == "precision" and isinstance(val, str):
            val = B.PRECISIONS[val]
        if key in _ARRAYS:
            vals = list(val) + [list(val)[-1]] * (_ARRAYS[key] - len(val))
            arr = getattr(p, key)
            for i in range(_ARRAYS[key]):
                arr[i] = int(vals[i])
        else:
            setattr(p, key, val)
    return p


class Solver:
    """A solver context on the current CUDA device.

    U: complex128 CUDA tensor (Lt, Lz, Ly, Lx, 4, 3, 3) of forward links.
    Keyword arguments are mg_params fields (precision may be 'fp64', 'fp32',
    'fp16', 'bf16'); ``init_vectors`` is an optional complex128 or complex64
    CUDA tensor of initial test vectors (N, Lt, Lz, Ly, Lx, 4, 3); ``setup2_start`` an optional
    complex128 CUDA tensor (coarse sites, 2N), the start vector of set-up part 2
    (used with ``setup2_iters`` > 0).
    """

    def __init__(self, U, c_sw, m0, init_vectors=None, setup2_start=None, stream=None, load=None, **params):
        if not (U.is_cuda and U.dtype == torch.complex128 and U.is_contiguous()):
            raise ValueError("U must be a contiguous complex128 CUDA tensor")
        lt, lz, ly, lx = U.shape[:4]
        self.dims = (lx, ly, lz, lt)
        self.lat = (lt, lz, ly, lx)
        self.params = make_params(self.dims, **params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params.stream = stream.cuda_stream
        self._init = None
        if init_vectors is not None:
            if init_vectors.dtype not in (torch.complex128, torch.complex64) or not init_vectors.is_cuda:
                raise ValueError("init_vectors must be a complex128 or complex64 CUDA tensor")
            self._init = init_vectors.contiguous()
            self.params.init_vectors = self._init.data_ptr()
            self.params.init_vectors_prec = B.MG_FP32 if init_vectors.dtype == torch.complex64 else B.MG_FP64
        self._start = None
        if setup2_start is not None:
            self._start = setup2_start.contiguous()
            self.params.setup2_start = self._start.data_ptr()
        self.prec = self.params.precision
        # load: a file written by save(); its test vectors replace the bootstrap set-up
        self.ctx = B.mg_setup(U, c_sw, m0, self.params) if load is None else \
            B.mg_setup_load(U, c_sw, m0, self.params, load)
        self._init = None
        self._start = None

    def spinor(self, nrhs=None, dtype=torch.complex128):
        shape = self.lat + (4, 3) if nrhs is None else (nrhs,) + self.lat + (4, 3)
        return torch.zeros(shape, dtype=dtype, device="cuda")

    def dirac(self, psi, prec=B.MG_FP64):
        nrhs = 1 if psi.dim() == 6 else psi.shape[0]
        out = torch.empty_like(psi)
        B.dirac_apply(self.ctx, psi, out, prec, nrhs)
        return out

    def smooth(self, b, z, n_sweeps):
        nrhs = 1 if b.dim() == 6 else b.shape[0]
        B.sap_smooth(self.ctx, b, z, n_sweeps, self.prec, nrhs)
        return z

    def solve(self, b):
        nrhs = 1 if b.dim() == 6 else b.shape[0]
        z = torch.empty_like(b)
        code, info = B.mg_solve(self.ctx, b, z, nrhs)
        return z, info, code

    def cgn_solve(self, b, tol=1e-10, maxiter=100000, prec=B.MG_FP64):
        """CG on the normal equations (the comparison method): (z, info, code)."""
        nrhs = 1 if b.dim() == 6 else b.shape[0]
        z = torch.empty_like(b)
        code, info = B.mg_cgn_solve(self.ctx, b, z, nrhs, prec, tol, maxiter)
        return z, info, code

    def history(self):
        """The last solve's residual history (mg_get_history) per right-hand side:
        {rhs: {"estimates": [(iteration, relres)], "fp64": [(iteration, relres)],
        "rho": the average residual reduction per iteration, (final relres)^(1/iterations)}}."""
        out = {}
        for it, q, r in B.mg_get_history(self.ctx):
            d = out.setdefault(q, {"estimates": [], "fp64": []})
            if it > 0:
                d["estimates"].append((it, r))
            else:
                d["fp64"].append((-it - 1, r))
        for d in out.values():
            k, r = d["fp64"][-1] if d["fp64"] else (0, 1.0)
            d["rho"] = r ** (1.0 / k) if k > 0 and r > 0 else None
        return out

    def save(self, path):
        """Write the set-up's test vectors to `path` (mg_save)."""
        B.mg_save(self.ctx, path)

    def close(self):
        if self.ctx is not None:
            B.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
