"""ctypes binding over the C ABI of include/nfl.h (libnfl.so).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are torch CUDA float64 tensors (torch provides device memory and the
current stream); blocks of right-hand sides are passed column-major.  There is
no CPU fallback: if the library is missing or a tensor is not on the GPU, the
call raises.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnfl.so")

NFL_OK = 0
NOALLOC_MAX_N = 262144   # NFL_NOALLOC_MAX_N in include/nfl.h
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32c": 2, "bf16w": 3}

_STATUS = {
    0: "NFL_OK", 1: "NFL_ERR_INVALID_ARG", 2: "NFL_ERR_NONPOSITIVE_DEGREE", 3: "NFL_ERR_BREAKDOWN",
    4: "NFL_ERR_NOT_CONVERGED", 5: "NFL_ERR_NAN", 6: "NFL_ERR_TIMEOUT", 7: "NFL_ERR_CUDA",
    8: "NFL_ERR_OUT_OF_MEMORY",
}


class NflError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        self.name = _STATUS.get(self.status, str(status))
        msg = _lib().nfl_status_string(self.status).decode() if _LIB is not None else self.name
        super().__init__("%s: %s (%s)" % (where, self.name, msg))


class Info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("d", ctypes.c_int), ("N", ctypes.c_int), ("m", ctypes.c_int),
        ("p", ctypes.c_int), ("precision", ctypes.c_int), ("sigma", ctypes.c_double),
        ("eps_B", ctypes.c_double), ("rho", ctypes.c_double), ("sigma_tilde", ctypes.c_double),
        ("center", ctypes.c_double * 3), ("box", ctypes.c_int * 3), ("tiles", ctypes.c_int64),
        ("work_items", ctypes.c_int64), ("min_degree", ctypes.c_double), ("max_degree", ctypes.c_double),
        ("degree_ok", ctypes.c_int), ("device_error", ctypes.c_int), ("kernel", ctypes.c_int),
        ("k0", ctypes.c_double), ("out_scale", ctypes.c_double),
        ("fft_lines_cap", ctypes.c_int), ("slide_tiles", ctypes.c_int), ("block_cols", ctypes.c_int),
        ("dense_items", ctypes.c_int64), ("chunk", ctypes.c_int), ("dense_cell", ctypes.c_int),
        ("dense_chunk", ctypes.c_int),
    ]


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64

SIGNATURES = {
    "nfl_plan_create": (_I, [_P, _L, _I, _I, _D, _I, _I, _I, _D, _I, _P, ctypes.POINTER(_P)]),
    "nfl_plan_create_batched": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_L), _I, _I, ctypes.POINTER(_D), _I, _I,
                                     _I, _D, _I, _P, ctypes.POINTER(_P)]),
    "nfl_plan_destroy": (None, [_P]),
    "nfl_plan_info": (_I, [_P, ctypes.POINTER(Info)]),
    "nfl_set_stream": (_I, [_P, _P]),
    "nfl_degree": (_I, [_P, _P]),
    "nfl_apply_W": (_I, [_P, _P, _L, _P, _L, _I]),
    "nfl_apply_A": (_I, [_P, _P, _L, _P, _L, _I]),
    "nfl_apply_Ls": (_I, [_P, _P, _L, _P, _L, _I]),
    "nfl_apply_host": (_I, [_P, _I, _P, _L, _P, _L, _I]),
    "nfl_lanczos_k_smallest": (_I, [_P, _I, _D, _I, ctypes.c_uint64, _P, _P, ctypes.POINTER(_I)]),
    "nfl_cg_solve": (_I, [_P, _D, _P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "nfl_apply_batched": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_P),
                               ctypes.POINTER(_L), _I]),
    "nfl_cg_solve_refined": (_I, [_P, _P, _D, _P, _P, _P, _D, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_D)]),
    "nfl_cg_solve_noalloc": (_I, [_P, _D, _P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "nfl_nystrom_k_largest": (_I, [_P, _I, _I, _I, _P, ctypes.c_uint64, _P, _P]),
    "nfl_form_grad_nodes": (_I, [_P, _P, _P, _P, _P]),
    "nfl_cg_solve_backward": (_I, [_P, _P, _D, _P, _P, _P, _D, _I, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                   ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "nfl_plan_autotune": (_I, [_P, ctypes.POINTER(_D)]),
    "nfl_plan_set_profiling": (_I, [_P, _I]),
    "nfl_plan_stage_times": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_L)]),
    "nfl_plan_kernels": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "nfl_plan_kernels_per_column": (_I, [_P, ctypes.POINTER(_I)]),
    "nfl_plan_inject_fault": (_I, [_P, _I]),
    "nfl_fma_rate": (_I, [_I, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "nfl_batch_create": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(_P), ctypes.POINTER(_L), ctypes.POINTER(_P),
                              ctypes.POINTER(_L), _I, _I, ctypes.POINTER(_P)]),
    "nfl_batch_parts": (_I, [_P, ctypes.POINTER(_I)]),
    "nfl_batch_run": (_I, [_P, _P]),
    "nfl_batch_destroy": (None, [_P]),
    "nfl_batch_set_profiling": (_I, [_P, _I]),
    "nfl_batch_stage_times": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_L)]),
    "nfl_status_string": (ctypes.c_char_p, [_I]),
}


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnfl.so is not built (%s); run paper_1808_04580_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _lib()


def _check(status, where):
    if status != NFL_OK:
        raise NflError(status, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _cuda_f64(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    return t


def _as_columns(x, n):
    """(n,) or (n, r) -> column-major (r, n) contiguous storage, r."""
    _cuda_f64(x, "x")
    if x.dim() == 1:
        if x.shape[0] != n:
            raise ValueError("x has %d rows, plan has %d" % (x.shape[0], n))
        return x.contiguous(), 1, True
    if x.dim() != 2 or x.shape[0] != n:
        raise ValueError("x must be (n,) or (n, r)")
    return x.t().contiguous(), x.shape[1], False


KERNELS = {"gaussian": 0, "laplacian_rbf": 1, "multiquadric": 2, "inverse_multiquadric": 3, "gaussian_dsigma": 4}


class Plan:
    """Alg. 2 setup for one point cloud; products with W, A and L_s.

    ``kernel`` names one of the kernels of Sec. 2 (``KERNELS``); ``sigma`` is its
    shape parameter (sigma, or c for the multiquadrics).
    """

    def __init__(self, v, sigma, N, m, p=0, eps_B=-1.0, precision="fp64", kernel="gaussian"):
        _cuda_f64(v, "v")
        if v.dim() != 2:
            raise ValueError("v must be (n, d)")
        v = v.contiguous()
        self.n, self.d = int(v.shape[0]), int(v.shape[1])
        self.device = v.device
        self._h = None
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = _lib().nfl_plan_create(v.data_ptr(), self.n, self.d, KERNELS[kernel], float(sigma), int(N), int(m), int(p),
                                        float(eps_B), PRECISIONS[precision], _stream(), ctypes.byref(h))
        _check(st, "nfl_plan_create")
        self._h = h

    @classmethod
    def _wrap(cls, handle, n, d, device):
        obj = cls.__new__(cls)
        obj.n, obj.d, obj.device, obj._h = int(n), int(d), device, handle
        return obj

    def close(self):
        if self._h is not None and _LIB is not None:
            _LIB.nfl_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = Info()
        _check(_lib().nfl_plan_info(self._h, ctypes.byref(inf)), "nfl_plan_info")
        out = {f: getattr(inf, f) for f, _ in Info._fields_}
        out["center"] = list(inf.center)
        out["box"] = list(inf.box)
        return out

    def autotune(self):
        """Time the plan's products under candidate launch parameters and keep the
        fastest (nfl_plan_autotune): dict(fft_lines_cap, slide_tiles, best_ms)."""
        self._sync_stream()
        ms = ctypes.c_double(0.0)
        _check(_lib().nfl_plan_autotune(self._h, ctypes.byref(ms)), "nfl_plan_autotune")
        inf = self.info()
        return dict(fft_lines_cap=inf["fft_lines_cap"], slide_tiles=inf["slide_tiles"], chunk=inf["chunk"],
                    dense_cell=inf["dense_cell"], dense_chunk=inf["dense_chunk"], best_ms=ms.value)

    def set_profiling(self, enable=True):
        _check(_lib().nfl_plan_set_profiling(self._h, 1 if enable else 0), "nfl_plan_set_profiling")

    def stage_times(self):
        """Accumulated ms per stage since the last call: dict(prep, spread, fft, gather, columns)."""
        ms = (ctypes.c_double * 4)()
        cols = ctypes.c_int64(0)
        _check(_lib().nfl_plan_stage_times(self._h, ms, ctypes.byref(cols)), "nfl_plan_stage_times")
        return dict(prep=ms[0], spread=ms[1], fft=ms[2], gather=ms[3], columns=cols.value)

    def inject_fault(self, kind):
        """Failure-detection test hook (nfl_plan_inject_fault)."""
        _check(_lib().nfl_plan_inject_fault(self._h, int(kind)), "nfl_plan_inject_fault")

    def kernels(self, nrhs=1):
        """Kernel launches one product of nrhs columns makes (nfl_plan_kernels)."""
        k = ctypes.c_int(0)
        _check(_lib().nfl_plan_kernels(self._h, int(nrhs), ctypes.byref(k)), "nfl_plan_kernels")
        return k.value

    def kernels_per_column(self):
        k = ctypes.c_int(0)
        _check(_lib().nfl_plan_kernels_per_column(self._h, ctypes.byref(k)), "nfl_plan_kernels_per_column")
        return k.value

    def _sync_stream(self):
        _check(_lib().nfl_set_stream(self._h, _stream()), "nfl_set_stream")

    def degree(self):
        self._sync_stream()
        d = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(_lib().nfl_degree(self._h, d.data_ptr()), "nfl_degree")
        return d

    def _apply(self, fn, name, x, out=None):
        self._sync_stream()
        xc, r, vec = _as_columns(x, self.n)
        y = torch.empty_like(xc) if out is None else out
        _check(fn(self._h, xc.data_ptr(), self.n, y.data_ptr(), self.n, r), name)
        return y if vec else y.t()

    def apply_W(self, x, out=None):
        """W_E x (Alg. 1 with W = W~ - K(0) I)."""
        return self._apply(_lib().nfl_apply_W, "nfl_apply_W", x, out)

    def apply_A(self, x, out=None):
        """A_E x (Alg. 2 step 5)."""
        return self._apply(_lib().nfl_apply_A, "nfl_apply_A", x, out)

    def apply_Ls(self, x, out=None):
        """L_s x = x - A_E x."""
        return self._apply(_lib().nfl_apply_Ls, "nfl_apply_Ls", x, out)

    def apply_host(self, x, op="Ls", out=None):
        """op(x) for a HOST float64 block, op in "W", "A", "Ls" (nfl_apply_host).

        x: CPU tensor (n,) or (n, r); the columns travel to the device and back
        in a pipeline that overlaps the copies with the products when x and out
        are in page-locked memory (``pin_memory()``).  Column-major storage, as
        ``X.t()`` of a contiguous (r, n) tensor, is used in place.  Returns a CPU
        tensor shaped like x (``out``: a contiguous (r, n) or (n,) CPU tensor).
        """
        if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.float64:
            raise TypeError("x must be a CPU float64 tensor")
        if x.dim() == 1:
            if x.shape[0] != self.n:
                raise ValueError("x has %d rows, plan has %d" % (x.shape[0], self.n))
            xc, r, vec = x.contiguous(), 1, True
        elif x.dim() == 2 and x.shape[0] == self.n:
            xc, r, vec = x.t().contiguous(), x.shape[1], False
        else:
            raise ValueError("x must be (n,) or (n, r)")
        if out is None:
            y = torch.empty_like(xc, pin_memory=xc.is_pinned())
        else:
            if out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != xc.numel():
                raise ValueError("out must be a contiguous CPU float64 tensor of r x n elements")
            y = out
        self._sync_stream()
        _check(_lib().nfl_apply_host(self._h, _OPS[op], xc.data_ptr(), self.n, y.data_ptr(), self.n, r),
               "nfl_apply_host")
        return y if vec else y.view(r, self.n).t()

    def lanczos_k_smallest(self, k, tol=1e-10, maxit=None, seed=0, vectors=True, check=True):
        """k smallest eigenpairs of L_s: (evals ndarray ascending, evecs (n, k) tensor or None, iters, status)."""
        self._sync_stream()
        if maxit is None:
            maxit = min(self.n, max(2 * k + 40, 60))
        evals = np.zeros(k, dtype=np.float64)
        evecs = torch.empty((k, self.n), dtype=torch.float64, device=self.device) if vectors else None
        iters = ctypes.c_int(0)
        st = _lib().nfl_lanczos_k_smallest(self._h, int(k), float(tol), int(maxit), int(seed),
                                           evals.ctypes.data, evecs.data_ptr() if vectors else None,
                                           ctypes.byref(iters))
        if check:
            _check(st, "nfl_lanczos_k_smallest")
        return evals, (evecs.t() if vectors else None), iters.value, st

    def nystrom_k_largest(self, k, L, M, G=None, seed=0, vectors=True):
        """Alg. 3: (eigenvalues of A descending (numpy), n x k vectors or None)."""
        self._sync_stream()
        gp = None
        if G is not None:
            G = _cuda_f64(G, "G")
            if G.shape != (self.n, L):
                raise ValueError("G must be (n, L)")
            G = G.t().contiguous()                   # column-major n x L
            gp = G.data_ptr()
        evals = np.zeros(k, dtype=np.float64)
        evecs = torch.empty((k, self.n), dtype=torch.float64, device=self.device) if vectors else None
        st = _lib().nfl_nystrom_k_largest(self._h, int(k), int(L), int(M), gp, int(seed), evals.ctypes.data,
                                          evecs.data_ptr() if vectors else None)
        _check(st, "nfl_nystrom_k_largest")
        return evals, (evecs.t() if vectors else None)

    def cg_solve(self, f, beta=1.0, shift=None, u0=None, tol=1e-10, maxit=1000, check=True, noalloc=False):
        """Solve (beta L_s + diag(shift)) u = f: (u, iters, relres, status).

        noalloc=True calls nfl_cg_solve_noalloc, whose scratch is a static
        device array (n <= NOALLOC_MAX_N) instead of per-call allocations.
        """
        self._sync_stream()
        _cuda_f64(f, "f")
        f = f.contiguous()
        u = torch.zeros_like(f) if u0 is None else _cuda_f64(u0, "u0").clone()
        sp = None
        if shift is not None:
            shift = _cuda_f64(shift, "shift").contiguous()
            sp = shift.data_ptr()
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        fn = _lib().nfl_cg_solve_noalloc if noalloc else _lib().nfl_cg_solve
        st = fn(self._h, float(beta), sp, f.data_ptr(), u.data_ptr(), float(tol), int(maxit),
                ctypes.byref(it), ctypes.byref(rel))
        if check:
            _check(st, "nfl_cg_solve_noalloc" if noalloc else "nfl_cg_solve")
        return u, it.value, rel.value, st

    def cg_solve_refined(self, inner, f, beta=1.0, shift=None, u0=None, tol=1e-10, inner_tol=1e-4, maxit=1000,
                         max_outer=10, check=True):
        """Solve (beta L_s + diag(shift)) u = f to this plan's accuracy with the correction
        solves on ``inner`` (nfl_cg_solve_refined): (u, inner_iters, outer_steps, relres, status)."""
        self._sync_stream()
        _cuda_f64(f, "f")
        f = f.contiguous()
        u = torch.zeros_like(f) if u0 is None else _cuda_f64(u0, "u0").clone()
        sp = None
        if shift is not None:
            shift = _cuda_f64(shift, "shift").contiguous()
            sp = shift.data_ptr()
        it, outer = ctypes.c_int(0), ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = _lib().nfl_cg_solve_refined(self._h, inner._h, float(beta), sp, f.data_ptr(), u.data_ptr(), float(tol),
                                         float(inner_tol), int(maxit), int(max_outer), ctypes.byref(it),
                                         ctypes.byref(outer), ctypes.byref(rel))
        if check:
            _check(st, "nfl_cg_solve_refined")
        return u, it.value, outer.value, rel.value, st

    def form_grad_nodes(self, v, a, b):
        """d(a^T A_E b)/dv for the nodes v (n, d) of this Gaussian plan (nfl_form_grad_nodes)."""
        self._sync_stream()
        v = _cuda_f64(v, "v").contiguous()
        a = _cuda_f64(a, "a").contiguous()
        b = _cuda_f64(b, "b").contiguous()
        if v.shape != (self.n, self.d) or a.shape != (self.n,) or b.shape != (self.n,):
            raise ValueError("v must be (n, d), a and b (n,)")
        g = torch.empty_like(v)
        _check(_lib().nfl_form_grad_nodes(self._h, v.data_ptr(), a.data_ptr(), b.data_ptr(), g.data_ptr()),
               "nfl_form_grad_nodes")
        return g

    def cg_solve_backward(self, u, g, beta=1.0, shift=None, dplan=None, tol=1e-10, maxit=1000, want_shift=True):
        """nfl_cg_solve_backward: (grad_f, grad_shift or None, grad_beta, grad_sigma or None, iters, relres)."""
        self._sync_stream()
        u = _cuda_f64(u, "u").contiguous()
        g = _cuda_f64(g, "g").contiguous()
        sp = None
        if shift is not None:
            shift = _cuda_f64(shift, "shift").contiguous()
            sp = shift.data_ptr()
        grad_f = torch.zeros_like(g)
        grad_shift = torch.empty_like(g) if want_shift else None
        gb = ctypes.c_double(0.0)
        gs = ctypes.c_double(0.0)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = _lib().nfl_cg_solve_backward(
            self._h, dplan._h if dplan is not None else None, float(beta), sp, u.data_ptr(), g.data_ptr(),
            float(tol), int(maxit), grad_f.data_ptr(), grad_shift.data_ptr() if want_shift else None,
            ctypes.byref(gb), ctypes.byref(gs) if dplan is not None else None, ctypes.byref(it), ctypes.byref(rel))
        _check(st, "nfl_cg_solve_backward")
        return grad_f, grad_shift, gb.value, (gs.value if dplan is not None else None), it.value, rel.value


_OPS = {"W": 0, "A": 1, "Ls": 2}


def create_batched(vs, sigma, N, m, p=0, eps_B=-1.0, precision="fp64", kernel="gaussian"):
    """Plans for a list of node sets in one library call (nfl_plan_create_batched).

    vs: list of (n_g, d) CUDA float64 tensors (same d); sigma: a number or one per
    set.  Returns the list of Plans, whose stream is the current stream.
    """
    G = len(vs)
    if G == 0:
        return []
    vs = [_cuda_f64(v, "v").contiguous() for v in vs]
    d = int(vs[0].shape[1])
    if any(v.dim() != 2 or v.shape[1] != d for v in vs):
        raise ValueError("every node set must be (n_g, d) with the same d")
    sig = [float(sigma)] * G if np.isscalar(sigma) else [float(s) for s in sigma]
    if len(sig) != G:
        raise ValueError("one sigma per node set")
    arr_v = (_P * G)(*[v.data_ptr() for v in vs])
    arr_n = (_L * G)(*[int(v.shape[0]) for v in vs])
    arr_s = (_D * G)(*sig)
    out = (_P * G)()
    with torch.cuda.device(vs[0].device):
        st = _lib().nfl_plan_create_batched(G, arr_v, arr_n, d, KERNELS[kernel], arr_s, int(N), int(m), int(p),
                                            float(eps_B), PRECISIONS[precision], _stream(), out)
    _check(st, "nfl_plan_create_batched")
    return [Plan._wrap(ctypes.c_void_p(out[g]), arr_n[g], d, vs[g].device) for g in range(G)]
RATE_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def fma_rate(kind="fp32"):
    """Measured multiply-add rate of the current device (nfl_fma_rate): (flop/s, ms)."""
    fl, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib().nfl_fma_rate(RATE_KINDS[kind], _stream(), ctypes.byref(fl), ctypes.byref(ms)), "nfl_fma_rate")
    return fl.value, ms.value


def apply_batched(plans, xs, op="Ls", outs=None):
    """op(x_g) for a batch of plans in one library call on the current stream.

    xs: list of (n_g,) or (n_g, r) CUDA float64 tensors (same r for all);
    returns the list of outputs.  The call issues no host synchronization, so
    it can be captured into a torch.cuda.CUDAGraph and replayed as one launch.
    """
    G = len(plans)
    if len(xs) != G:
        raise ValueError("one right-hand side block per plan")
    cols, ys, vecs, nrhs = [], [], [], None
    for g, (plan, x) in enumerate(zip(plans, xs)):
        xc, r, vec = _as_columns(x, plan.n)
        if nrhs is None:
            nrhs = r
        elif r != nrhs:
            raise ValueError("every block needs the same number of columns")
        cols.append(xc)
        ys.append(torch.empty_like(xc) if outs is None else outs[g])
        vecs.append(vec)
    for plan in plans:
        plan._sync_stream()
    arr_p = (_P * G)(*[p._h for p in plans])
    arr_x = (_P * G)(*[c.data_ptr() for c in cols])
    arr_y = (_P * G)(*[y.data_ptr() for y in ys])
    arr_l = (_L * G)(*[p.n for p in plans])
    _check(_lib().nfl_apply_batched(arr_p, G, _OPS[op], arr_x, arr_y, arr_l, int(nrhs or 1)), "nfl_apply_batched")
    return [y if v else y.t() for y, v in zip(ys, vecs)]


class Batch:
    """Products of many plans with one launch per stage and part (nfl_batch_create / nfl_batch_run).

    plans: Plans of one mixed precision, m and N (3-D), split into ``parts`` groups
    that run concurrently; xs: their (n_g,) or (n_g, r)
    CUDA float64 blocks (same r), bound at creation together with the outputs
    (``outs``: contiguous (r, n_g) or (n_g,) tensors, else allocated).  ``run()``
    issues the products on the current stream (capturable in a CUDA graph);
    ``outputs`` are shaped like xs.  Column-major x blocks (``X.t()`` of a
    contiguous (r, n) tensor) are used in place, so they can be refilled between runs.
    """

    def __init__(self, plans, xs, op="Ls", outs=None, parts=1):
        G = len(plans)
        if len(xs) != G or G == 0:
            raise ValueError("one block per plan")
        cols, ys, vecs, nrhs = [], [], [], None
        for g, (plan, x) in enumerate(zip(plans, xs)):
            xc, r, vec = _as_columns(x, plan.n)
            if nrhs is None:
                nrhs = r
            elif r != nrhs:
                raise ValueError("every block needs the same number of columns")
            cols.append(xc)
            ys.append(torch.empty_like(xc) if outs is None else outs[g])
            vecs.append(vec)
        self._plans, self._x, self._y, self._vec = list(plans), cols, ys, vecs
        self._h = None
        arr_p = (_P * G)(*[p._h for p in plans])
        arr_x = (_P * G)(*[c.data_ptr() for c in cols])
        arr_y = (_P * G)(*[y.data_ptr() for y in ys])
        arr_l = (_L * G)(*[p.n for p in plans])
        h = ctypes.c_void_p()
        _check(_lib().nfl_batch_create(arr_p, G, _OPS[op], arr_x, arr_l, arr_y, arr_l, int(nrhs), int(parts),
                                       ctypes.byref(h)), "nfl_batch_create")
        self._h = h
        k = ctypes.c_int(0)
        _check(_lib().nfl_batch_parts(self._h, ctypes.byref(k)), "nfl_batch_parts")
        self.parts = k.value

    def run(self):
        _check(_lib().nfl_batch_run(self._h, _stream()), "nfl_batch_run")
        return self.outputs

    @property
    def outputs(self):
        return [y if v else y.t() for y, v in zip(self._y, self._vec)]

    def set_profiling(self, enable=True):
        _check(_lib().nfl_batch_set_profiling(self._h, 1 if enable else 0), "nfl_batch_set_profiling")

    def stage_times(self):
        """Accumulated ms per stage since the last call: dict(prep, spread, fft, gather, runs)."""
        ms = (ctypes.c_double * 4)()
        runs = ctypes.c_int64(0)
        _check(_lib().nfl_batch_stage_times(self._h, ms, ctypes.byref(runs)), "nfl_batch_stage_times")
        return dict(prep=ms[0], spread=ms[1], fft=ms[2], gather=ms[3], runs=runs.value)

    def close(self):
        if self._h is not None and _LIB is not None:
            _LIB.nfl_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
