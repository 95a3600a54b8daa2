"""GB300 (sm_103a) CVS-ADC(2) hot path: Python front end of libcvsadc.

The package is a thin layer over the C ABI of ``include/cvsadc.h``: it
marshals numpy arrays (host memory) or torch CUDA tensors (device memory)
into the library calls.  All arithmetic runs in the library's CUDA
kernels; importing :class:`Context` fails loudly when the library is not
built.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    CVSADC_FLAG_DEVICE_PTRS, CVSADC_FLAG_DIAG_PRECOND, CVSADC_FLAG_FOLDED,
    CVSADC_FLAG_NO_REFINE, CVSADC_FLAG_RETURN_X,
    CVSADC_FP64, CVSADC_MIXED_BF16X3, CVSADC_ENOTCONV, Info, Params,
)

PRECISIONS = {"fp64": CVSADC_FP64, "bf16x3": CVSADC_MIXED_BF16X3,
              "slice4": 2, "fp64_slice7": 3}


class CvsadcError(RuntimeError):
    def __init__(self, code, text):
        super().__init__("cvsadc error %d: %s" % (code, text))
        self.code = code


def _is_torch_cuda(x):
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and x.is_cuda


def _ptr(x):
    """(pointer, is_device) of a numpy array or torch CUDA tensor."""
    if x is None:
        return None, None
    if _is_torch_cuda(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), True
    if not isinstance(x, np.ndarray) or not x.flags.c_contiguous:
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    return ctypes.c_void_p(x.ctypes.data), False


def _inputs_ready(*xs):
    """The library reads device inputs on its own stream without waiting on
    torch's: finish the work torch has queued on the producing stream."""
    for x in xs:
        if _is_torch_cuda(x):
            import torch
            torch.cuda.current_stream(x.device).synchronize()
            return


class Context:
    """One libcvsadc context (one device, one stream)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream)) if stream else None
        rc = self.lib.cvsadc_create(ctypes.byref(h), device, s)
        if rc != 0:
            raise CvsadcError(rc, self.lib.cvsadc_strerror(rc).decode())
        self.h = h
        self._shape = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.cvsadc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow_notconv=False):
        if rc == 0 or (allow_notconv and rc == CVSADC_ENOTCONV):
            return rc
        msg = self.lib.cvsadc_last_error(self.h).decode() or \
            self.lib.cvsadc_strerror(rc).decode()
        raise CvsadcError(rc, msg)

    # ------------------------------------------------------------ params
    @staticmethod
    def params(ncore, nval, nvirt, naux, nroots=4, precision="fp64",
               tau=0.0, conv=1e-6, max_iter=0, max_subspace=0, flags=0,
               refine_sweeps=0):
        p = Params()
        p.ncore, p.nval, p.nvirt, p.naux = ncore, nval, nvirt, naux
        p.nroots = nroots
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        p.fns_threshold = tau
        p.conv_residual = conv
        p.max_iter = max_iter
        p.max_subspace = max_subspace
        p.flags = flags
        p.refine_sweeps = refine_sweeps
        return p

    # ----------------------------------------------------------- stages
    def prepare(self, eps, B, dip=None, ncore=None, nval=None, nvirt=None,
                precision="fp64", tau=0.0):
        naux = B.shape[0]
        _inputs_ready(eps, B, dip)
        pe, dev = _ptr(eps)
        pb, _ = _ptr(B)
        pd, _ = _ptr(dip)
        p = self.params(ncore, nval, nvirt, naux, 1, precision, tau,
                        flags=CVSADC_FLAG_DEVICE_PTRS if dev else 0)
        info = Info()
        self._check(self.lib.cvsadc_prepare(self.h, ctypes.byref(p), pe, pb, pd,
                                            ctypes.byref(info)))
        nv = ctypes.c_int32()
        n1 = ctypes.c_int64()
        n2 = ctypes.c_int64()
        self._check(self.lib.cvsadc_prepared_sizes(self.h, ctypes.byref(nv),
                                                   ctypes.byref(n1), ctypes.byref(n2)))
        self._shape = dict(ncore=ncore, nval=nval, nvirt_in=nvirt, nvirt=nv.value,
                           naux=naux, N1=n1.value, N2=n2.value, N=n1.value + n2.value)
        return info.as_dict()

    @property
    def shape(self):
        return self._shape

    def get_t2(self):
        s = self._shape
        o = s["ncore"] + s["nval"]
        v = s["nvirt"]
        t2 = np.empty((o, o, v, v), dtype=np.complex128)
        e = ctypes.c_double()
        self._check(self.lib.cvsadc_get_t2(self.h, 0, ctypes.c_void_p(t2.ctypes.data),
                                           ctypes.byref(e)))
        return t2, e.value

    def get_m11(self):
        n1 = self._shape["N1"]
        m = np.empty((n1, n1), dtype=np.complex128)
        self._check(self.lib.cvsadc_get_m11(self.h, 0, ctypes.c_void_p(m.ctypes.data)))
        return m

    def get_schur(self, theta):
        """S(theta) = M11 + M12 (theta - M22)^-1 M21 of the prepared problem."""
        n1 = self._shape["N1"]
        S = np.empty((n1, n1), dtype=np.complex128)
        self._check(self.lib.cvsadc_get_schur(self.h, ctypes.c_double(theta), 0,
                                              ctypes.c_void_p(S.ctypes.data)))
        return S

    def get_moments(self):
        F = np.empty((3, self._shape["N"]), dtype=np.complex128)
        self._check(self.lib.cvsadc_get_moments(self.h, 0, ctypes.c_void_p(F.ctypes.data)))
        return F

    def get_fns(self):
        s = self._shape
        occ = np.empty(s["nvirt_in"], dtype=np.float64)
        U = np.empty((s["nvirt_in"], s["nvirt"]), dtype=np.complex128)
        self._check(self.lib.cvsadc_get_fns(self.h, 0, ctypes.c_void_p(occ.ctypes.data),
                                            ctypes.c_void_p(U.ctypes.data)))
        return occ, U

    def sigma(self, x, precision="fp64", out=None):
        """sigma = M x for x [nvec][N] (numpy host or torch CUDA)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        nvec = x.shape[0] if x.ndim == 2 else 1
        _inputs_ready(x)
        px, dev = _ptr(x)
        if out is None:
            if dev:
                import torch
                out = torch.empty_like(x)
            else:
                out = np.empty_like(x)
        po, _ = _ptr(out)
        flags = CVSADC_FLAG_DEVICE_PTRS if dev else 0
        self._check(self.lib.cvsadc_sigma(self.h, prec, flags, px, po, nvec))
        return out

    def wait_probe(self, limit_ns):
        """Run one bounded device wait that nothing satisfies (limit clamped
        to [1 ms, 4 s]); raises CvsadcError(CVSADC_ETIMEOUT) when it expires
        as designed.  The context stays usable."""
        self._check(self.lib.cvsadc_wait_probe(self.h, int(limit_ns)))

    def zgemm(self, A, B, precision="fp64"):
        """C = A B (complex) with the library's GEMM engines."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        M, K = A.shape
        K2, N = B.shape
        assert K == K2
        _inputs_ready(A, B)
        pa, dev = _ptr(A)
        pb, _ = _ptr(B)
        if dev:
            import torch
            C = torch.empty((M, N), dtype=A.dtype, device=A.device)
        else:
            C = np.empty((M, N), dtype=np.complex128)
        pc, _ = _ptr(C)
        flags = CVSADC_FLAG_DEVICE_PTRS if dev else 0
        self._check(self.lib.cvsadc_zgemm(self.h, prec, flags, M, N, K, pa, K, pb, N,
                                          pc, N))
        return C

    def spectrum(self, omega, osc, e0_ev, de_ev, npts, fwhm_ev=0.3, shift_ev=0.0):
        """Lorentzian-broadened spectrum (numpy [npts]) of roots omega (Eh)
        and oscillator strengths osc on the grid e0_ev + g de_ev."""
        w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        f = np.ascontiguousarray(np.asarray(osc, dtype=np.float64))
        out = np.empty(int(npts))
        self._check(self.lib.cvsadc_spectrum(
            self.h, 0, w.size, ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(f.ctypes.data),
            float(e0_ev), float(de_ev), int(npts), float(fwhm_ev), float(shift_ev),
            ctypes.c_void_p(out.ctypes.data)))
        return out

    def block_dot(self, A, B, precision="fp64"):
        """A^H B (numpy [ma][mb]) of torch CUDA blocks A [ma][N], B [mb][N]
        in the Davidson solver's arithmetic for `precision`."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        _inputs_ready(A, B)
        pa, dev = _ptr(A)
        pb, _ = _ptr(B)
        if not dev:
            raise ValueError("block_dot takes device tensors")
        out = np.empty((A.shape[0], B.shape[0]), dtype=np.complex128)
        self._check(self.lib.cvsadc_block_dot(self.h, prec, pa, A.shape[0], pb,
                                              B.shape[0], A.shape[1],
                                              ctypes.c_void_p(out.ctypes.data)))
        return out

    def davidson(self, nroots, precision="fp64", conv=1e-6, max_iter=0,
                 max_subspace=0, return_x=False, refine=True, precond="schur",
                 solver="auto"):
        s = self._shape
        flags = (CVSADC_FLAG_DIAG_PRECOND if precond == "diag" else 0) | \
            (CVSADC_FLAG_RETURN_X if return_x else 0) | \
            (0 if refine else CVSADC_FLAG_NO_REFINE) | \
            (CVSADC_FLAG_FOLDED if solver == "folded" else 0)
        p = self.params(s["ncore"], s["nval"], s["nvirt"], s["naux"], nroots,
                        precision, 0.0, conv, max_iter, max_subspace, flags)
        omega = np.empty(nroots)
        osc = np.empty(nroots)
        X = np.empty((nroots, s["N"]), dtype=np.complex128) if return_x else None
        info = Info()
        rc = self.lib.cvsadc_davidson(
            self.h, ctypes.byref(p), ctypes.c_void_p(omega.ctypes.data),
            ctypes.c_void_p(X.ctypes.data) if X is not None else None,
            ctypes.c_void_p(osc.ctypes.data), ctypes.byref(info))
        self._check(rc, allow_notconv=True)
        return dict(omega=omega, osc=osc, X=X, info=info.as_dict(), status=rc)

    def grad(self, eps, B, ncore, nval, nvirt, nroots, root_mask=None, conv=1e-8,
             max_iter=0, precision="fp64"):
        """(roots, dE/deps, dE/dB) for E = sum of the selected roots, through
        cvsadc_grad (FP64 problem, root solve in `precision` with FP64-class
        refinement, FP64 adjoint pass).  Host numpy or torch CUDA."""
        naux = B.shape[0]
        _inputs_ready(eps, B)
        pe, dev = _ptr(eps)
        pb, _ = _ptr(B)
        p = self.params(ncore, nval, nvirt, naux, nroots, precision, 0.0, conv,
                        max_iter, 0, CVSADC_FLAG_DEVICE_PTRS if dev else 0)
        mask = None if root_mask is None else np.ascontiguousarray(root_mask, dtype=np.int32)
        if dev:
            import torch
            omega = torch.empty(nroots, dtype=torch.float64, device=eps.device)
            ge = torch.empty_like(eps)
            gB = torch.empty_like(B)
        else:
            omega = np.empty(nroots)
            ge = np.empty_like(eps)
            gB = np.empty_like(B)
        rc = self.lib.cvsadc_grad(self.h, ctypes.byref(p), pe, pb,
                                  ctypes.c_void_p(mask.ctypes.data) if mask is not None else None,
                                  _ptr(omega)[0], _ptr(ge)[0], _ptr(gB)[0])
        self._check(rc)
        return omega, ge, gB

    def solve(self, eps, B, dip, ncore, nval, nvirt, nroots, precision="fp64",
              tau=0.0, conv=1e-6, max_iter=0, max_subspace=0, return_x=False,
              refine=True, refine_sweeps=0, precond="schur", solver="auto"):
        """The whole path through cvsadc_solve.  solver: "auto" (the library
        picks), or "folded" (the doubles-folded solver)."""
        naux = B.shape[0]
        _inputs_ready(eps, B, dip)
        pe, dev = _ptr(eps)
        pb, _ = _ptr(B)
        pd, _ = _ptr(dip)
        flags = (CVSADC_FLAG_DEVICE_PTRS if dev else 0) | \
            (CVSADC_FLAG_RETURN_X if return_x else 0) | \
            (0 if refine else CVSADC_FLAG_NO_REFINE) | \
            (CVSADC_FLAG_DIAG_PRECOND if precond == "diag" else 0) | \
            (CVSADC_FLAG_FOLDED if solver == "folded" else 0)
        p = self.params(ncore, nval, nvirt, naux, nroots, precision, tau, conv,
                        max_iter, max_subspace, flags, refine_sweeps)
        if dev:
            import torch
            omega = torch.empty(nroots, dtype=torch.float64, device=eps.device)
            osc = torch.empty(nroots, dtype=torch.float64, device=eps.device)
        else:
            omega = np.empty(nroots)
            osc = np.empty(nroots)
        X = None
        if return_x:
            # the size after FNS truncation is known only after the call;
            # the untruncated space bounds it
            nv = nvirt
            N = ncore * nv + ncore * nval * nv * (nv - 1) // 2
            X = np.zeros(nroots * N, dtype=np.complex128)
        info = Info()
        rc = self.lib.cvsadc_solve(
            self.h, ctypes.byref(p), pe, pb, pd, _ptr(omega)[0],
            ctypes.c_void_p(X.ctypes.data) if X is not None else None,
            _ptr(osc)[0] if dip is not None else None, ctypes.byref(info))
        self._check(rc, allow_notconv=True)
        nv = ctypes.c_int32()
        n1 = ctypes.c_int64()
        n2 = ctypes.c_int64()
        self._check(self.lib.cvsadc_prepared_sizes(self.h, ctypes.byref(nv),
                                                   ctypes.byref(n1), ctypes.byref(n2)))
        self._shape = dict(ncore=ncore, nval=nval, nvirt_in=nvirt, nvirt=nv.value,
                           naux=naux, N1=n1.value, N2=n2.value, N=n1.value + n2.value)
        if X is not None:
            X = X[: nroots * self._shape["N"]].reshape(nroots, self._shape["N"])
        return dict(omega=omega, osc=osc if dip is not None else None, X=X,
                    info=info.as_dict(), status=rc)

    def device_bytes(self):
        """Bytes the context's device buffers hold (cvsadc_device_bytes)."""
        out = ctypes.c_int64()
        self._check(self.lib.cvsadc_device_bytes(self.h, ctypes.byref(out)))
        return out.value

    def solve_batched(self, instances, nroots, precision="fp64", tau=0.0, conv=1e-6,
                      max_iter=0, return_x=False, refine=True, lanes=0):
        """Independent problems through cvsadc_solve_batched.  `instances` is
        a list of dicts with eps, B, dip (may be None), ncore, nval, nvirt
        (numpy host arrays or torch CUDA tensors).  Returns one dict per
        instance (omega, osc, X, info, status)."""
        n = len(instances)
        params = (Params * n)()
        infos = (Info * n)()
        keep, outs = [], []
        ptrs = {k: (ctypes.c_void_p * n)() for k in ("eps", "B", "dip", "omega", "X", "osc")}
        any_dip = False
        for i, inst in enumerate(instances):
            eps, B, dip = inst["eps"], inst["B"], inst.get("dip")
            _inputs_ready(eps, B, dip)
            pe, dev = _ptr(eps)
            pb, _ = _ptr(B)
            pd, _ = _ptr(dip)
            nc, nw, nv = inst["ncore"], inst["nval"], inst["nvirt"]
            flags = (CVSADC_FLAG_DEVICE_PTRS if dev else 0) | \
                (CVSADC_FLAG_RETURN_X if return_x else 0) | \
                (0 if refine else CVSADC_FLAG_NO_REFINE)
            params[i] = self.params(nc, nw, nv, B.shape[0], nroots, precision, tau, conv,
                                    max_iter, 0, flags)
            if dev:
                import torch
                omega = torch.empty(nroots, dtype=torch.float64, device=eps.device)
                osc = torch.empty(nroots, dtype=torch.float64, device=eps.device)
            else:
                omega, osc = np.empty(nroots), np.empty(nroots)
            X = None
            if return_x:
                N = nc * nv + nc * nw * nv * (nv - 1) // 2
                X = np.zeros(nroots * N, dtype=np.complex128)
            ptrs["eps"][i], ptrs["B"][i] = pe, pb
            ptrs["dip"][i] = pd
            any_dip = any_dip or dip is not None
            ptrs["omega"][i] = _ptr(omega)[0]
            ptrs["osc"][i] = _ptr(osc)[0] if dip is not None else None
            ptrs["X"][i] = ctypes.c_void_p(X.ctypes.data) if X is not None else None
            keep.append((eps, B, dip))
            outs.append((omega, osc if dip is not None else None, X, N if return_x else 0))
        status = np.zeros(n, dtype=np.int32)
        rc = self.lib.cvsadc_solve_batched(
            self.h, n, params, ptrs["eps"], ptrs["B"], ptrs["dip"] if any_dip else None,
            ptrs["omega"], ptrs["X"] if return_x else None, ptrs["osc"] if any_dip else None,
            infos, ctypes.c_void_p(status.ctypes.data), lanes)
        self._check(rc, allow_notconv=True)
        res = []
        for i, (omega, osc, X, N) in enumerate(outs):
            if X is not None:
                X = X.reshape(nroots, N)
            res.append(dict(omega=omega, osc=osc, X=X, info=infos[i].as_dict(),
                            status=int(status[i])))
        return res


def estimate_bytes(ncore, nval, nvirt, naux, nroots=4, precision="fp64", tau=0.0,
                   max_subspace=0, solver="auto"):
    """cvsadc_estimate_bytes: device bytes one solve holds at its peak (host
    arithmetic, no GPU needed); solver="folded" prices the doubles-folded
    solver."""
    lib = _lib.load()
    p = Context.params(ncore, nval, nvirt, naux, nroots, precision, tau,
                       max_subspace=max_subspace,
                       flags=CVSADC_FLAG_FOLDED if solver == "folded" else 0)
    out = ctypes.c_int64()
    rc = lib.cvsadc_estimate_bytes(ctypes.byref(p), ctypes.byref(out))
    if rc != 0:
        raise CvsadcError(rc, lib.cvsadc_strerror(rc).decode())
    return out.value


def energy_function(ctx, ncore, nval, nvirt, nroots, precision="fp64", conv=1e-8):
    """A torch.autograd.Function: E(eps, B) = sum of the lowest nroots
    CVS-ADC(2) roots, with the gradient from the library's adjoint pass
    (cvsadc_grad).  eps and B are torch CUDA tensors (B complex128)."""
    import torch

    class CVSADCEnergy(torch.autograd.Function):
        @staticmethod
        def forward(fctx, eps, B):
            # the adjoint pass runs only when a gradient can be asked for
            if fctx.needs_input_grad[0] or fctx.needs_input_grad[1]:
                omega, ge, gB = ctx.grad(eps.contiguous(), B.contiguous(), ncore, nval,
                                         nvirt, nroots, conv=conv, precision=precision)
                fctx.save_for_backward(ge, gB)
                return omega.sum()
            out = ctx.solve(eps.contiguous(), B.contiguous(), None, ncore, nval, nvirt,
                            nroots, precision=precision, conv=conv)
            return torch.as_tensor(out["omega"], device=eps.device).sum()

        @staticmethod
        def backward(fctx, gE):
            ge, gB = fctx.saved_tensors
            return gE * ge, gE * gB

    return CVSADCEnergy
