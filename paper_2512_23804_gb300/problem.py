"""Thin Python front end over the C ABI: device memory and streams come from
PyTorch, every computation runs in the CUDA library (libsgoc.so)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import abi

_PREC = {"fp64": abi.SGOC_FP64, "mixed": abi.SGOC_MIXED_FP32}


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class SGProblem:
    """One SG optimal-control problem (Sec. 2 steady / Sec. 3 all-at-once time).

    Host arrays follow include/sgoc.h: kappa (M+1, nx, nx) element values with
    kappa[0] the (constant) mean, yhat (max(nt,1), n) target values at interior
    nodes, y0 (n,) or None.
    """

    def __init__(self, nx, M, p, kappa, beta, yhat, gamma=0.0, nt=0, T=1.0, y0=None, *, tol=1e-8,
                 max_iter=1000, r=0, cheb_steps=5, nu=2, omega=0.8, precision="fp64", inner_tol=1e-4,
                 max_outer=20):
        self._handle = None
        lib = abi.load()
        self._kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        self._yhat = np.ascontiguousarray(yhat, dtype=np.float64)
        self._y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None
        desc = abi.ProblemDesc(nx, M, p, dp(self._kappa), beta, gamma, nt, T, dp(self._yhat), dp(self._y0))
        opts = abi.Options()
        lib.sgoc_default_options(ctypes.byref(opts))
        opts.tol, opts.max_iter, opts.r, opts.cheb_steps = tol, max_iter, r, cheb_steps
        opts.nu_pre = opts.nu_post = nu
        opts.omega, opts.precision = omega, _PREC[precision]
        opts.inner_tol, opts.max_outer = inner_tol, max_outer
        h = ctypes.c_void_p()
        abi.check(lib.sgoc_problem_create(ctypes.byref(desc), ctypes.byref(opts), ctypes.byref(h)),
                  "sgoc_problem_create")
        self._handle = h
        n, P, S, N = (ctypes.c_int64() for _ in range(4))
        abi.check(lib.sgoc_problem_sizes(h, ctypes.byref(n), ctypes.byref(P), ctypes.byref(S), ctypes.byref(N)),
                  "sgoc_problem_sizes")
        self.n, self.P, self.slabs, self.kkt_size = n.value, P.value, S.value, N.value
        self.nx, self.M, self.p, self.nt = nx, M, p, nt
        self.precision = precision
        pers, ws = ctypes.c_size_t(), ctypes.c_size_t()
        abi.check(lib.sgoc_problem_device_bytes(h, ctypes.byref(pers), ctypes.byref(ws)), "device_bytes")
        self.persistent_bytes, self.workspace_bytes = pers.value, ws.value
        self._persistent = None
        self._ws = None

    @classmethod
    def from_problem(cls, pr, **kw):
        """Build from any object with the attributes of a problem instance
        (nx, M, p, kappa, beta, gamma, nt, T, yhat, y0, tol, max_iter, r, cheb_steps,
        nu_pre, omega)."""
        r = getattr(pr, "r", -1)
        args = dict(gamma=pr.gamma, nt=pr.nt, T=pr.T, y0=pr.y0, tol=pr.tol, max_iter=pr.max_iter,
                    r=0 if r is None or r < 0 else r, cheb_steps=pr.cheb_steps, nu=pr.nu_pre, omega=pr.omega)
        args.update(kw)
        return cls(pr.nx, pr.M, pr.p, pr.kappa, pr.beta, pr.yhat, **args)

    def __del__(self):
        if getattr(self, "_handle", None) is not None:
            try:
                abi.load().sgoc_problem_destroy(self._handle)
            except Exception:
                pass
            self._handle = None

    # ---- device side -------------------------------------------------------
    def upload(self, stream=None):
        import torch
        lib = abi.load()
        if self._persistent is None:
            self._persistent = torch.empty(max(self.persistent_bytes, 256), dtype=torch.uint8, device="cuda")
            abi.check(lib.sgoc_problem_upload(self._handle, _dptr(self._persistent), self.persistent_bytes,
                                              _stream(stream)), "sgoc_problem_upload")
        return self

    def workspace(self):
        import torch
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
        return self._ws

    def release_workspace(self):
        self._ws = None

    def rhs(self, stream=None):
        import torch
        self.upload(stream)
        b = torch.empty(self.kkt_size, dtype=torch.float64, device="cuda")
        abi.check(abi.load().sgoc_rhs(self._handle, _dptr(b), _stream(stream)), "sgoc_rhs")
        return b

    def solve(self, x0=None, out=None, stream=None):
        import torch
        self.upload(stream)
        ws = self.workspace()
        x = out if out is not None else torch.empty(self.kkt_size, dtype=torch.float64, device="cuda")
        res = abi.Result()
        st = abi.load().sgoc_solve(self._handle, _dptr(ws), ws.numel(), _dptr(x0) if x0 is not None else None,
                                   _dptr(x), _stream(stream), ctypes.byref(res))
        info = res.as_dict()
        info["status_name"] = abi.STATUS_NAMES.get(st, st)
        if st != abi.SGOC_OK:
            raise abi.SgocError(st, f"sgoc_solve {info}")
        return x, info

    def _prec_id(self, t):
        import torch
        return 0 if t.dtype == torch.float64 else 1

    def apply_operator(self, X, nslabs=1, out=None, stream=None):
        import torch
        self.upload(stream)
        Y = out if out is not None else torch.empty_like(X)
        abi.check(abi.load().sgoc_apply_operator(self._handle, self._prec_id(X), _dptr(X), _dptr(Y), nslabs,
                                                 _stream(stream)), "sgoc_apply_operator")
        return Y

    def apply_kkt(self, v, out=None, stream=None):
        import torch
        self.upload(stream)
        w = out if out is not None else torch.empty_like(v)
        abi.check(abi.load().sgoc_apply_kkt(self._handle, self._prec_id(v), _dptr(v), _dptr(w), _stream(stream)),
                  "sgoc_apply_kkt")
        return w

    def _prec_ws(self, dtype):
        import torch
        # the solve workspace of either precision contains a preconditioner workspace of
        # that precision; for the hooks size a dedicated one generously (the solve size)
        ws = self.workspace()
        return ws

    def apply_precond(self, r, out=None, stream=None):
        import torch
        self.upload(stream)
        z = out if out is not None else torch.empty_like(r)
        ws = self._prec_ws(r.dtype)
        abi.check(abi.load().sgoc_apply_precond(self._handle, self._prec_id(r), _dptr(r), _dptr(z), _dptr(ws),
                                                ws.numel(), _stream(stream)), "sgoc_apply_precond")
        return z

    def apply_hgs(self, R, nslabs=None, out=None, stream=None):
        import torch
        self.upload(stream)
        V = out if out is not None else torch.empty_like(R)
        ws = self._prec_ws(R.dtype)
        ns = self.slabs if nslabs is None else nslabs
        abi.check(abi.load().sgoc_apply_hgs(self._handle, self._prec_id(R), _dptr(R), _dptr(V), ns, _dptr(ws),
                                            ws.numel(), _stream(stream)), "sgoc_apply_hgs")
        return V

    def apply_vcycle(self, R, ncols, out=None, stream=None):
        import torch
        self.upload(stream)
        X = out if out is not None else torch.empty_like(R)
        ws = self._prec_ws(R.dtype)
        abi.check(abi.load().sgoc_apply_vcycle(self._handle, self._prec_id(R), _dptr(R), _dptr(X), ncols, _dptr(ws),
                                               ws.numel(), _stream(stream)), "sgoc_apply_vcycle")
        return X

    def apply_chebyshev(self, R, ncols, out=None, stream=None):
        import torch
        self.upload(stream)
        X = out if out is not None else torch.empty_like(R)
        ws = self._prec_ws(R.dtype)
        abi.check(abi.load().sgoc_apply_chebyshev(self._handle, self._prec_id(R), _dptr(R), _dptr(X), ncols,
                                                  _dptr(ws), ws.numel(), _stream(stream)), "sgoc_apply_chebyshev")
        return X

    # ---- host-side tables ----------------------------------------------------
    def pc_indices(self):
        out = np.zeros((self.P, max(self.M, 1)), dtype=np.int32)
        abi.check(abi.load().sgoc_pc_indices(self._handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
                  "sgoc_pc_indices")
        return out[:, :self.M]

    def triple_products(self):
        lib = abi.load()
        nnz = ctypes.c_int64(0)
        abi.check(lib.sgoc_triple_products(self._handle, None, None, None, None, ctypes.byref(nnz)), "tp count")
        k = np.zeros(nnz.value, np.int32)
        a = np.zeros(nnz.value, np.int32)
        b = np.zeros(nnz.value, np.int32)
        c = np.zeros(nnz.value, np.float64)
        pi = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        abi.check(lib.sgoc_triple_products(self._handle, pi(k), pi(a), pi(b),
                                           c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(nnz)),
                  "sgoc_triple_products")
        return k, a, b, c
