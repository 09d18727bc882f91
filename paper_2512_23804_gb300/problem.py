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

    def __init__(self, nx, M, p, kappa, beta, yhat, gamma=0.0, nt=0, T=1.0, y0=None, *, chaos="legendre",
                 length=1.0, tol=1e-8,
                 max_iter=1000, r=0, cheb_steps=5, nu=2, omega=0.8, precision="fp64", inner_tol=1e-3,
                 max_outer=20, schur="diagonal", krylov="minres", restart=64, mass_solve="chebyshev",
                 precond="block", mean_solve="vcycle"):
        self._handle = None
        lib = abi.load()
        self._kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        self._yhat = np.ascontiguousarray(yhat, dtype=np.float64)
        self._y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None
        desc = abi.ProblemDesc(nx, M, p, dp(self._kappa), beta, gamma, nt, T, dp(self._yhat), dp(self._y0),
                               {"legendre": 0, "hermite": 1}[chaos], length)
        opts = abi.Options()
        lib.sgoc_default_options(ctypes.byref(opts))
        opts.tol, opts.max_iter, opts.r, opts.cheb_steps = tol, max_iter, r, cheb_steps
        opts.nu_pre = opts.nu_post = nu
        opts.omega, opts.precision = omega, _PREC[precision]
        opts.inner_tol, opts.max_outer = inner_tol, max_outer
        opts.schur = {"diagonal": 0, "coupled": 1}[schur]
        opts.krylov = {"minres": 0, "fgmres": 1}[krylov]
        opts.restart = restart
        opts.mass_solve = {"chebyshev": 0, "exact": 1}[mass_solve]
        opts.precond = {"block": 0, "hgsoc": 1}[precond]
        opts.mean_solve = {"vcycle": 0, "exact": 1}[mean_solve]
        if precond == "hgsoc":
            opts.krylov = 1                   # the hGSoc preconditioner is not symmetric
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
                    r=0 if r is None or r < 0 else r, cheb_steps=pr.cheb_steps, nu=pr.nu_pre, omega=pr.omega,
                    schur=getattr(pr, "schur", "diagonal"), krylov=getattr(pr, "krylov", "minres"),
                    mass_solve=getattr(pr, "mass_solve", "chebyshev"), precond=getattr(pr, "precond", "block"),
                    chaos=getattr(pr, "chaos", "legendre"), length=getattr(pr, "length", 1.0),
                    restart=getattr(pr, "restart", 64), mean_solve=getattr(pr, "mean_solve", "vcycle"))
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

    def autotune(self, stream=None):
        """Time the SG kernel variants on this problem's launch shapes and keep the
        fastest per shape (process-wide); returns the chosen kernel per shape."""
        self.upload(stream)
        ws = self.workspace()
        n = 2 * self.p + 4
        chosen = (ctypes.c_int32 * n)()
        abi.check(abi.load().sgoc_autotune(self._handle, _dptr(ws), ws.numel(), ctypes.cast(chosen, ctypes.c_void_p),
                                           n, _stream(stream)), "sgoc_autotune")
        return list(chosen)

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

    def set_kernel(self, shape, variant, precision=None):
        """Pin SG kernel `variant` (-1: built-in rule) for launch shape `shape` (0 KKT,
        1 operator, 2 + d return visit of hGS level d, 3 + p + d first visit of level d)
        in this problem's precision (or the given one)."""
        prec = precision if precision is not None else (0 if self.precision == "fp64" else 1)
        abi.check(abi.load().sgoc_set_kernel(self._handle, prec, shape, variant), "sgoc_set_kernel")

    def apply_operator_variant(self, X, variant, nslabs=1, out=None, stream=None):
        """The SG operator with a given kernel variant (0..7, see sgoc_autotune)."""
        import torch
        self.upload(stream)
        Y = out if out is not None else torch.empty_like(X)
        abi.check(abi.load().sgoc_apply_operator_variant(self._handle, self._prec_id(X), variant, _dptr(X), _dptr(Y),
                                                         nslabs, _stream(stream)), "sgoc_apply_operator_variant")
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


def solve_batch(problems, x0s=None, outs=None, streams=None, merged=False):
    """Solve several SGProblem instances concurrently (sgoc_solve_batch): each on its
    own CUDA stream, all advanced together by the calling thread; with merged=True
    (sgoc_solve_batch_merged) problems of one shape share merged SG and V-cycle
    launches in lockstep iterations.  Returns ([x_i], [info_i])."""
    import torch
    lib = abi.load()
    n = len(problems)
    for sp in problems:
        sp.upload()
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(n)]
    # the caller's current stream must not race with the solve streams
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    xs = outs if outs is not None else [torch.empty(sp.kkt_size, dtype=torch.float64, device="cuda")
                                        for sp in problems]
    wss = [sp.workspace() for sp in problems]
    P = ctypes.c_void_p
    arr = lambda vals: (P * n)(*vals)
    res = (abi.Result * n)()
    fn = lib.sgoc_solve_batch_merged if merged else lib.sgoc_solve_batch
    st = fn(
        n, arr([sp._handle.value for sp in problems]), arr([w.data_ptr() for w in wss]),
        (ctypes.c_size_t * n)(*[w.numel() for w in wss]),
        arr([(x0.data_ptr() if x0 is not None else None) for x0 in x0s]) if x0s is not None else None,
        arr([x.data_ptr() for x in xs]), arr([s.cuda_stream for s in streams]), res)
    for s in streams:
        cur.wait_stream(s)
    infos = []
    for r in res:
        d = r.as_dict()
        d["status_name"] = abi.STATUS_NAMES.get(r.status, r.status)
        infos.append(d)
    if st != abi.SGOC_OK:
        raise abi.SgocError(st, f"sgoc_solve_batch {infos}")
    return xs, infos


class SGServer:
    """Continuous-batching solve server (sgoc_server_*) over a device pool taken
    from PyTorch.  submit() queues a problem; step() runs one sweep; poll()
    returns finished (request_id, solution tensor, info)."""

    def __init__(self, pool_bytes, max_active=8):
        import torch
        lib = abi.load()
        self._pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        abi.check(lib.sgoc_server_create(_dptr(self._pool), pool_bytes, max_active, ctypes.byref(h)),
                  "sgoc_server_create")
        self._h = h
        self._pending = {}

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            try:
                abi.load().sgoc_server_destroy(self._h)
            except Exception:
                pass
            self._h = None

    def submit(self, sp, request_id):
        import torch
        x = torch.empty(sp.kkt_size, dtype=torch.float64, device="cuda")
        torch.cuda.current_stream().synchronize()
        abi.check(abi.load().sgoc_server_submit(self._h, sp._handle, _dptr(x), ctypes.c_uint64(request_id)),
                  "sgoc_server_submit")
        sp._persistent = None                 # the server uploads into its pool
        self._pending[request_id] = (sp, x)

    def step(self):
        na, nq = ctypes.c_int32(), ctypes.c_int32()
        abi.check(abi.load().sgoc_server_step(self._h, ctypes.byref(na), ctypes.byref(nq)), "sgoc_server_step")
        return na.value, nq.value

    def poll(self, cap=64):
        ids = (ctypes.c_uint64 * cap)()
        res = (abi.Result * cap)()
        n = ctypes.c_int32()
        abi.check(abi.load().sgoc_server_poll(self._h, ids, res, cap, ctypes.byref(n)), "sgoc_server_poll")
        out = []
        for i in range(n.value):
            sp, x = self._pending.pop(ids[i])
            d = res[i].as_dict()
            d["status_name"] = abi.STATUS_NAMES.get(res[i].status, res[i].status)
            out.append((ids[i], x, d))
        return out

    def stats(self):
        a, c, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        hw = ctypes.c_size_t()
        abi.check(abi.load().sgoc_server_stats(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(r),
                                               ctypes.byref(hw)), "sgoc_server_stats")
        return dict(admitted=a.value, completed=c.value, rejected=r.value, pool_high_water=hw.value)

    @property
    def pending(self):
        return len(self._pending)
