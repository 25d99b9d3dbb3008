"""Python binding of liblogdet.so with the C-ABI's names.

Argument marshalling only: tensors must already be on the GPU (torch owns
device memory and streams); every step of the computation runs in the
library's CUDA kernels.  Blocks of vectors are row-major n-by-c tensors.
"""
import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import LdKernel, LdOptions, LdResult, check

RBF = _lib.RBF
MATERN52 = _lib.MATERN52
PRECISIONS = _lib.PRECISIONS


@dataclass
class Kernel:
    """k(r) with r = |x - y|; RBF: v exp(-r^2/(2 l^2)); Matern-5/2: v (1+u+u^2/3) e^-u,
    u = sqrt(5) r / l.  noise is added to the diagonal of K."""
    kind: int
    lengthscale: float
    variance: float = 1.0
    noise: float = 0.0

    def c(self):
        return LdKernel(int(self.kind), 0, float(self.lengthscale), float(self.variance), float(self.noise))


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensor must be on a CUDA device")
        if t is not None and not t.is_contiguous():
            raise ValueError("tensor must be contiguous")


def _points(X):
    _need_cuda(X)
    if X.dtype != torch.float64 or X.dim() != 2:
        raise ValueError("X must be an n-by-d float64 CUDA tensor")
    return X


def _workspace(nbytes, device):
    if nbytes == 0:
        return None, 0
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device), int(nbytes)


def rk_coeffs(order):
    """(b, c, sigma) of Table 1's partial fractions, from the library."""
    lib = _lib.load()
    b = ctypes.c_double()
    c = (ctypes.c_double * 5)()
    s = (ctypes.c_double * 5)()
    check(lib.ld_rk_coeffs(order, ctypes.byref(b), c, s), "ld_rk_coeffs")
    return b.value, np.array(c[:order]), np.array(s[:order])


def ld_kz(X, V, kernel, precision="fp32", out=None, stream=None):
    """W = (K(X, X) + noise I) V."""
    lib = _lib.load()
    X = _points(X)
    p = _prec(precision)
    want = torch.float64 if p == _lib.FP64 else torch.float32
    _need_cuda(V)
    if V.dtype != want or V.dim() != 2 or V.shape[0] != X.shape[0]:
        raise ValueError("V must be n-by-c %s" % want)
    W = torch.empty_like(V) if out is None else out
    n, d = X.shape
    c = V.shape[1]
    ws, nb = _workspace(lib.ld_kz_workspace_size(n, d, c, p), X.device)
    check(lib.ld_kz(_ptr(X), n, d, kernel.c(), _ptr(V), _ptr(W), c, p, _ptr(ws), nb, _stream(stream)),
          "ld_kz")
    return W


def ld_kz_dl(X, V, kernel, precision="fp32", stream=None):
    """(K V, dK/dl V) without the noise term."""
    lib = _lib.load()
    X = _points(X)
    p = _prec(precision)
    want = torch.float64 if p == _lib.FP64 else torch.float32
    _need_cuda(V)
    if V.dtype != want or V.dim() != 2 or V.shape[0] != X.shape[0]:
        raise ValueError("V must be n-by-c %s" % want)
    W = torch.empty_like(V)
    Wdl = torch.empty_like(V)
    n, d = X.shape
    check(lib.ld_kz_dl(_ptr(X), n, d, kernel.c(), _ptr(V), _ptr(W), _ptr(Wdl), V.shape[1], p,
                       _stream(stream)), "ld_kz_dl")
    return W, Wdl


def ld_dense_materialize(X, kernel, precision="fp32", stream=None):
    """M = K(X, X) + noise I as a dense n-by-n tensor (float64 for fp64, else float32)."""
    lib = _lib.load()
    X = _points(X)
    p = _prec(precision)
    n, d = X.shape
    M = torch.empty((n, n), dtype=torch.float64 if p == _lib.FP64 else torch.float32, device=X.device)
    check(lib.ld_dense_materialize(_ptr(X), n, d, kernel.c(), p, _ptr(M), _stream(stream)), "ld_dense_materialize")
    return M


def ld_dense_kz(M, V, precision="fp32", stream=None):
    """W = M V for a stored dense M (n-by-n; float64 for fp64, else float32; positive
    semidefinite for the tensor-core precisions, as every K + noise I is)."""
    lib = _lib.load()
    want = torch.float64 if _prec(precision) == _lib.FP64 else torch.float32
    if M.dtype != want or M.dim() != 2 or M.shape[0] != M.shape[1]:
        raise ValueError("M must be an n-by-n %s tensor" % want)
    if V.dtype != want or V.dim() != 2 or V.shape[0] != M.shape[0]:
        raise ValueError("V must be an n-by-c %s tensor" % want)
    _need_cuda(M, V)
    W = torch.empty_like(V)
    check(lib.ld_dense_kz(_ptr(M), M.shape[0], _ptr(V), _ptr(W), V.shape[1], _prec(precision), _stream(stream)),
          "ld_dense_kz")
    return W


def ld_gaussian(seed, n, s, col0=0, device="cuda", stream=None):
    """n-by-s float64 N(0,1) block (Box-Muller over SplitMix64(seed))."""
    lib = _lib.load()
    Z = torch.empty((n, s), dtype=torch.float64, device=device)
    check(lib.ld_gaussian(seed, n, s, col0, _ptr(Z), _stream(stream)), "ld_gaussian")
    return Z


def ld_rademacher(seed, n, s, col0=0, device="cuda", stream=None):
    """n-by-s int8 Rademacher block from SplitMix64(seed)."""
    lib = _lib.load()
    Z = torch.empty((n, s), dtype=torch.int8, device=device)
    check(lib.ld_rademacher(seed, n, s, col0, _ptr(Z), _stream(stream)), "ld_rademacher")
    return Z


class Precond:
    """Owner of an ld_precond handle (P = D + A A^T and its split factor)."""

    def __init__(self, handle, precision):
        self._h = handle
        self.precision = precision
        lib = _lib.load()
        n = ctypes.c_int64()
        r = ctypes.c_int32()
        pr = ctypes.c_int32()
        ld = ctypes.c_double()
        check(lib.precond_info(self._h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(pr),
                               ctypes.byref(ld)), "precond_info")
        self.n, self.rank, self.logdet_P = n.value, r.value, ld.value

    @classmethod
    def build(cls, X, kernel, rank, power_iters=2, seed=2, precision="fp32", stream=None):
        lib = _lib.load()
        X = _points(X)
        p = _prec(precision)
        n, d = X.shape
        ws, nb = _workspace(lib.precond_workspace_size(n, d, rank, p), X.device)
        h = ctypes.c_void_p()
        check(lib.precond_build(_ptr(X), n, d, kernel.c(), rank, power_iters, seed, p, _ptr(ws), nb,
                                _stream(stream), ctypes.byref(h)), "precond_build")
        return cls(h, p)

    @classmethod
    def build_scaled(cls, X, kernel, rank, a, power_iters=2, seed=2, precision="fp32", stream=None):
        """P = a I + A A^T (Appendix "plus scaling")."""
        lib = _lib.load()
        X = _points(X)
        p = _prec(precision)
        n, d = X.shape
        ws, nb = _workspace(lib.precond_workspace_size(n, d, rank, p), X.device)
        h = ctypes.c_void_p()
        check(lib.precond_build_scaled(_ptr(X), n, d, kernel.c(), rank, power_iters, seed, float(a), p, _ptr(ws),
                                       nb, _stream(stream), ctypes.byref(h)), "precond_build_scaled")
        return cls(h, p)

    @classmethod
    def import_(cls, A, D, precision="fp32", stream=None):
        lib = _lib.load()
        A = np.ascontiguousarray(A, dtype=np.float64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        n, r = A.shape
        h = ctypes.c_void_p()
        check(lib.precond_import(A.ctypes.data_as(ctypes.c_void_p), D.ctypes.data_as(ctypes.c_void_p),
                                 n, r, _prec(precision), _stream(stream), ctypes.byref(h)),
              "precond_import")
        return cls(h, _prec(precision))

    def export(self, stream=None):
        lib = _lib.load()
        A = np.zeros((self.n, self.rank))
        D = np.zeros(self.n)
        ld = ctypes.c_double()
        check(lib.precond_export(self._h, A.ctypes.data_as(ctypes.c_void_p),
                                 D.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ld), _stream(stream)),
              "precond_export")
        return A, D, ld.value

    def apply(self, V, transpose=False, stream=None):
        """L^-1 V (or L^-T V): V is n-by-c, float64 for an fp64 handle, else float32."""
        lib = _lib.load()
        want = torch.float64 if self.precision == _lib.FP64 else torch.float32
        if V.dtype != want or V.dim() != 2 or V.shape[0] != self.n:
            raise ValueError("V must be an n-by-c %s tensor" % want)
        _need_cuda(V)
        W = torch.empty_like(V)
        check(lib.precond_apply(self._h, int(transpose), _ptr(V), _ptr(W), V.shape[1], _stream(stream)),
              "precond_apply")
        return W

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            _lib.load().precond_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_options(order=3, num_probes=16, probes_per_block=None, max_iters=1000, fixed_iters=0,
                 precision="fp32", residual_check=False, seed=1, rel_tol=1e-6, dense=False, probe_kind="rademacher",
                 probe_col0=0):
    kind = {"rademacher": 0, "gaussian": 1, "orthogonal": 2}[probe_kind] if isinstance(probe_kind, str) else int(probe_kind)
    return LdOptions(int(order), int(num_probes), int(probes_per_block or num_probes), int(max_iters),
                     int(fixed_iters), _prec(precision), int(bool(residual_check)), int(bool(dense)), int(seed),
                     float(rel_tol), kind, int(probe_col0))


def ld_combine(brackets, logdet_P):
    """Algorithm 1's output (log det, trace, std-err) from per-probe brackets (host)."""
    lib = _lib.load()
    br = np.ascontiguousarray(brackets, dtype=np.float64)
    res = LdResult()
    check(lib.ld_combine(br.ctypes.data_as(ctypes.c_void_p), int(br.size), float(logdet_P), ctypes.byref(res)),
          "ld_combine")
    return {"logdet": res.logdet, "logdet_P": res.logdet_P, "trace_est": res.trace_est, "std_err": res.std_err}


def _result_dict(res, status, per_probe=None):
    out = {
        "logdet": res.logdet, "logdet_P": res.logdet_P, "trace_est": res.trace_est,
        "std_err": res.std_err, "iters": res.iters, "converged": bool(res.converged),
        "max_resid": list(res.max_resid), "final_rel_resid": res.final_rel_resid, "status": status,
        "slq_logdet": res.slq_logdet,
    }
    if per_probe is not None:
        out["per_probe"] = per_probe
    return out


def logdet_estimate(X, kernel, precond=None, probes=None, stream=None, ws=None, allow_not_converged=False,
                    **opts):
    """Run the estimator; returns a dict with the ld_result fields and per-probe brackets."""
    lib = _lib.load()
    X = _points(X)
    o = make_options(**opts)
    n, d = X.shape
    if probes is not None:
        _need_cuda(probes)
        if probes.dtype != torch.int8 or tuple(probes.shape) != (n, o.num_probes):
            raise ValueError("probes must be an n-by-num_probes int8 CUDA tensor")
    ph = precond.handle if precond is not None else None
    if ws is None:
        ws, nb = _workspace(lib.logdet_workspace_size(n, d, ph, ctypes.byref(o)), X.device)
    else:
        nb = ws.numel()
    res = LdResult()
    pp = np.zeros(o.num_probes)
    st = lib.logdet_estimate(_ptr(X), n, d, kernel.c(), ph, ctypes.byref(o), _ptr(probes),
                             pp.ctypes.data_as(ctypes.c_void_p), _ptr(ws), nb, _stream(stream),
                             ctypes.byref(res))
    if not (allow_not_converged and st == _lib.LD_ERR_NOT_CONVERGED):
        check(st, "logdet_estimate")
    return _result_dict(res, st, pp)


def logdet_grad(X, kernel, precond=None, probes=None, stream=None, allow_not_converged=False, **opts):
    """Estimate and its gradient w.r.t. (lengthscale, variance, noise), P and probes frozen."""
    lib = _lib.load()
    X = _points(X)
    o = make_options(**opts)
    n, d = X.shape
    ph = precond.handle if precond is not None else None
    ws, nb = _workspace(lib.logdet_workspace_size(n, d, ph, ctypes.byref(o)), X.device)
    res = LdResult()
    g = (ctypes.c_double * 3)()
    st = lib.logdet_grad(_ptr(X), n, d, kernel.c(), ph, ctypes.byref(o), _ptr(probes), _ptr(ws), nb,
                         _stream(stream), g, ctypes.byref(res))
    if not (allow_not_converged and st == _lib.LD_ERR_NOT_CONVERGED):
        check(st, "logdet_grad")
    out = _result_dict(res, st)
    out["grad"] = np.array(g[:])
    return out


N_SURROGATE_PARAMS = 33793


class Surrogate:
    """Owner of an ld_surrogate handle: the 4-128-128-128-1 GELU MLP that maps
    (log lengthscale, log variance, log noise, log n) to log det / n."""

    def __init__(self, seed=0, stream=None):
        lib = _lib.load()
        h = ctypes.c_void_p()
        check(lib.surrogate_create(seed, _stream(stream), ctypes.byref(h)), "surrogate_create")
        self._h = h

    def set_params(self, flat, stream=None):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == N_SURROGATE_PARAMS
        check(_lib.load().surrogate_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "surrogate_set_params")

    def get_params(self, stream=None):
        flat = np.zeros(N_SURROGATE_PARAMS, dtype=np.float32)
        check(_lib.load().surrogate_get_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "surrogate_get_params")
        return flat

    def get_norm(self, stream=None):
        norm = np.zeros(10, dtype=np.float32)
        check(_lib.load().surrogate_get_norm(self._h, norm.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "surrogate_get_norm")
        return norm

    def set_norm(self, norm, stream=None):
        norm = np.ascontiguousarray(norm, dtype=np.float32)
        assert norm.size == 10
        check(_lib.load().surrogate_set_norm(self._h, norm.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "surrogate_set_norm")

    def save(self, path):
        """Checkpoint: parameters and normalisation to an .npz file."""
        np.savez(path, params=self.get_params(), norm=self.get_norm())

    def load(self, path):
        """Restore a checkpoint written by save()."""
        with np.load(path) as z:
            self.set_params(z["params"])
            self.set_norm(z["norm"])

    @staticmethod
    def _f32(t, cols):
        _need_cuda(t)
        if t.dtype != torch.float32:
            raise ValueError("surrogate tensors are float32")
        if cols and (t.dim() != 2 or t.shape[1] != cols):
            raise ValueError("expected N-by-%d" % cols)
        return t

    def loss_grad(self, theta, y, stream=None):
        self._f32(theta, 4)
        self._f32(y, 0)
        loss = ctypes.c_double()
        g = np.zeros(N_SURROGATE_PARAMS, dtype=np.float32)
        check(_lib.load().surrogate_loss_grad(self._h, _ptr(theta), _ptr(y), theta.shape[0], ctypes.byref(loss),
                                              g.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
              "surrogate_loss_grad")
        return loss.value, g

    def train(self, theta, y, epochs, batch, lr=1e-3, stream=None):
        self._f32(theta, 4)
        self._f32(y, 0)
        loss = ctypes.c_double()
        check(_lib.load().surrogate_train(self._h, _ptr(theta), _ptr(y), theta.shape[0], epochs, batch,
                                          ctypes.c_float(lr), _stream(stream), ctypes.byref(loss)),
              "surrogate_train")
        return loss.value

    def infer(self, q, want_grad=False, stream=None):
        self._f32(q, 4)
        out = torch.empty(q.shape[0], dtype=torch.float32, device=q.device)
        dout = torch.empty_like(q) if want_grad else None
        check(_lib.load().surrogate_infer(self._h, _ptr(q), q.shape[0], _ptr(out), _ptr(dout), _stream(stream)),
              "surrogate_infer")
        return (out, dout) if want_grad else out

    def free(self):
        if self._h is not None and self._h.value:
            _lib.load().surrogate_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
