"""Tensor-level wrapper around one solver handle (``sylv_create`` ... ``sylv_destroy``).

The wrapper only moves inputs to the device in the layouts ``include/sylv.h`` documents and
calls the C ABI; all arithmetic runs in the library's kernels.
"""

import numpy as np

from . import binding as B


def _to_device(x, dtype, device):
    import torch
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


class Operator:
    """G = sum_j (e_j e_j^T) kron tau_j (kappa_j^2 W + L) + sum_c (a_c a_c^T) kron D_c
    (prior="igmrf": L^2 in place of L, the intrinsic GMRF of App. C).

    Vectors are torch tensors of shape (R, k, ld) or (k, ld) (float64 unless noted)."""

    def __init__(self, *, rowptr, col, val, D, tau, kappa, nu=None, beta=None, A=None, w=None,
                 ld=None, nu0=0.0, prior="gmrf", device="cuda", stream=None):
        import torch
        self.device = torch.device(device)
        D = _to_device(D, torch.float64, self.device)
        self.m = int(D.shape[0])
        n = int(np.asarray(rowptr).shape[0] - 1) if not isinstance(rowptr, torch.Tensor) \
            else int(rowptr.numel() - 1)
        self.n = n
        self.ld = int(ld) if ld is not None else n
        if D.dim() != 2 or D.shape[1] < self.n:
            raise ValueError("D must be (m, >= n)")
        if D.shape[1] != self.ld:
            Dp = torch.zeros((self.m, self.ld), dtype=torch.float64, device=self.device)
            Dp[:, :self.n] = D[:, :self.n]
            D = Dp
        self.k = int(np.asarray(tau).reshape(-1).shape[0])
        self._rowptr = _to_device(rowptr, torch.int32, self.device)
        self._col = _to_device(col, torch.int32, self.device)
        self._val = _to_device(val, torch.float64, self.device)
        self._w = _to_device(w, torch.float64, self.device) if w is not None else None
        self._D = D
        self.tau = np.asarray(tau, dtype=np.float64).reshape(-1)
        self.kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
        self.nu = None if nu is None else np.asarray(nu, dtype=np.float64).reshape(-1)
        self.beta = None if beta is None else np.asarray(beta, dtype=np.float64).reshape(-1)
        self.A = None if A is None else np.asarray(A, dtype=np.float64).reshape(self.m, self.k)
        self.handle = B.sylv_create(n=self.n, k=self.k, m=self.m, ld=self.ld,
                                    L_rowptr=self._rowptr, L_col=self._col, L_val=self._val,
                                    D=self._D, tau=self.tau, kappa=self.kappa, nu=self.nu,
                                    beta=self.beta, A=self.A, w=self._w, nu0=nu0,
                                    prior={"gmrf": B.SYLV_PRIOR_GMRF,
                                           "igmrf": B.SYLV_PRIOR_IGMRF}[prior],
                                    stream=stream)

    # -- helpers ---------------------------------------------------------------------------
    def zeros(self, nrhs=1, dtype=None):
        import torch
        return torch.zeros((nrhs, self.k, self.ld), dtype=dtype or torch.float64,
                           device=self.device)

    def _batch(self, X, rows):
        X = X if X.dim() == 3 else X.unsqueeze(0)
        if X.shape[1] != rows or X.shape[2] != self.ld:
            raise ValueError(f"expected (R, {rows}, {self.ld}), got {tuple(X.shape)}")
        return X.contiguous()

    def close(self):
        if getattr(self, "handle", None):
            B.sylv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points --------------------------------------------------------------------------
    def rhs(self, Yobs, stream=None):
        """b = B^T C y for Yobs (R, m, ld) -> (R, k, ld)."""
        import torch
        Y = self._batch(Yobs.to(torch.float64), self.m)
        out = torch.empty((Y.shape[0], self.k, self.ld), dtype=torch.float64, device=self.device)
        B.sylv_rhs(self.handle, Y, out, Y.shape[0], k=self.k, m=self.m, ld=self.ld, n=self.n,
                   stream=stream)
        return out

    def apply(self, X, stream=None):
        """Y = G X in the dtype of X (float32 or float64)."""
        import torch
        Xb = self._batch(X, self.k)
        Y = torch.empty_like(Xb)
        B.sylv_apply(self.handle, Xb, Y, Xb.shape[0], k=self.k, ld=self.ld, n=self.n,
                     stream=stream)
        return Y

    def residual(self, Bv, X, stream=None):
        """R = B - G X (float64 (R, k, ld)), as the mixed-precision solve forms it."""
        import torch
        Bb = self._batch(Bv.to(torch.float64), self.k)
        Xb = self._batch(X.to(torch.float64), self.k)
        out = torch.empty_like(Bb)
        B.sylv_residual(self.handle, Bb, Xb, out, Bb.shape[0], k=self.k, ld=self.ld, n=self.n,
                        stream=stream)
        return out

    def solve(self, Bv, X0=None, *, opts=None, stream=None, allow_not_converged=False,
              allow=(), **kw):
        """X = G^{-1} B; returns (X, info dict)."""
        Bb = self._batch(Bv, self.k)
        if opts is None:
            opts = B.make_opts(**kw)
        # without a start the library zeroes X itself (the whole nrhs x k x ld block)
        X = Bb.new_empty(Bb.shape) if X0 is None else self._batch(X0, self.k).clone()
        opts.use_x0 = 1 if X0 is not None else 0
        allow = tuple(allow) + ((B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ())
        code, info = B.sylv_solve(self.handle, Bb, X, Bb.shape[0], opts, k=self.k, ld=self.ld,
                                  n=self.n, stream=stream, allow=allow)
        d = info.as_dict()
        d["code"] = code
        return X, d

    def solve_host(self, Yobs, X0=None, *, out=None, opts=None, stream=None,
                   allow_not_converged=False, allow=(), **kw):
        """Posterior mean from host observations: Yobs (nrhs, m, ld) float64 on the host
        (page-locked for overlapped copies); returns (X on the host (nrhs, k, ld), info).  The
        copies run inside the call, overlapping the computation (sylv_solve_host)."""
        import torch
        Yb = Yobs if Yobs.dim() == 3 else Yobs.unsqueeze(0)
        nrhs = Yb.shape[0]
        if opts is None:
            opts = B.make_opts(**kw)
        if out is None:
            out = torch.empty((nrhs, self.k, self.ld), dtype=torch.float64).pin_memory()
        if X0 is not None:
            out.copy_(X0 if X0.dim() == 3 else X0.unsqueeze(0))
            opts.use_x0 = 1
        allow = tuple(allow) + ((B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ())
        code, info = B.sylv_solve_host(self.handle, Yb, out, nrhs, opts, k=self.k, m=self.m,
                                       ld=self.ld, n=self.n, stream=stream, allow=allow)
        d = info.as_dict()
        d["code"] = code
        return out, d

    def solve_sylvester(self, Bv, X0=None, *, opts=None, stream=None,
                        allow_not_converged=False, allow=(), **kw):
        """X = G^{-1} B through the Sylvester form and block Lanczos (separable noise, one
        prior shape); returns (X, info dict)."""
        Bb = self._batch(Bv, self.k)
        if opts is None:
            opts = B.make_opts(**kw)
        # without a start the library zeroes X itself (the whole nrhs x k x ld block)
        X = Bb.new_empty(Bb.shape) if X0 is None else self._batch(X0, self.k).clone()
        opts.use_x0 = 1 if X0 is not None else 0
        allow = tuple(allow) + ((B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ())
        code, info = B.sylv_solve_sylvester(self.handle, Bb, X, Bb.shape[0], opts, k=self.k,
                                            ld=self.ld, n=self.n, stream=stream, allow=allow)
        d = info.as_dict()
        d["code"] = code
        return X, d

    def variance(self, Z, *, opts=None, stream=None, allow_not_converged=False, **kw):
        """Posterior variances diag(G^{-1}) (k, ld) estimated from the probes Z (S, k, ld)."""
        Zb = self._batch(Z, self.k)
        if opts is None:
            opts = B.make_opts(**kw)
        var = Zb.new_zeros((self.k, self.ld))
        allow = (B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ()
        code, info = B.sylv_variance(self.handle, Zb, Zb.shape[0], var, opts, k=self.k,
                                     ld=self.ld, n=self.n, stream=stream, allow=allow)
        d = info.as_dict()
        d["code"] = code
        return var, d

    def variance_probing(self, colour, ncolours, *, opts=None, stream=None,
                         allow_not_converged=False, **kw):
        """Posterior variances diag(G^{-1}) (k, ld) from the probing vectors of a pixel
        colouring (colour: n integers in [0, ncolours))."""
        import torch
        col = _to_device(colour, torch.int32, self.device)
        if opts is None:
            opts = B.make_opts(**kw)
        var = torch.zeros((self.k, self.ld), dtype=torch.float64, device=self.device)
        allow = (B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ()
        code, info = B.sylv_variance_probing(self.handle, col, int(ncolours), var, opts,
                                             k=self.k, ld=self.ld, n=self.n, stream=stream,
                                             allow=allow)
        d = info.as_dict()
        d["code"] = code
        return var, d

    def set_params(self, tau, kappa, *, nu=None, beta=None, A=None, stream=None):
        """New prior scalars and mixing for this handle (sylv_set_params)."""
        tau = np.asarray(tau, dtype=np.float64).reshape(-1)
        kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
        if A is None:
            nu = self.nu if nu is None else np.asarray(nu, dtype=np.float64).reshape(-1)
            beta = self.beta if beta is None else np.asarray(beta, dtype=np.float64).reshape(-1)
        B.sylv_set_params(self.handle, k=self.k, m=self.m, tau=tau, kappa=kappa, nu=nu,
                          beta=None if A is not None else beta, A=A, stream=stream)
        self.tau, self.kappa = tau, kappa
        if A is None:
            self.nu, self.beta, self.A = nu, beta, None
        else:
            self.A = np.asarray(A, dtype=np.float64).reshape(self.m, self.k)

    def backward(self, Xhat, dLdX, Yobs=None, *, opts=None, want=("tau", "kappa", "beta"),
                 stream=None, lam0=None, **kw):
        """Gradients (g_tau, g_kappa, g_beta) of a loss with dl/dX = dLdX at X = Xhat.  lam0: an
        earlier adjoint solution to start the adjoint solve from (warm start)."""
        Xb = self._batch(Xhat, self.k)
        Gb = self._batch(dLdX, self.k)
        Yb = self._batch(Yobs, self.m) if Yobs is not None else None
        if opts is None:
            opts = B.make_opts(**kw)
        if lam0 is not None:
            lam = self._batch(lam0, self.k).clone()
            opts.use_x0 = 1
        else:
            lam = Xb.new_empty(Xb.shape)      # zeroed by the library (no start given)
            opts.use_x0 = 0
        gt, gk, gb, info = B.sylv_backward(self.handle, Xb, Gb, Yb, Xb.shape[0], lam, opts,
                                           k=self.k, m=self.m, ld=self.ld, n=self.n,
                                           want=want, stream=stream)
        return gt, gk, gb, lam, info.as_dict()


def solve_batched(ops, Bs, *, opts=None, stream=None, allow_not_converged=False, **kw):
    """Solves several Operators' systems in one batched call.  Returns (Xs, infos)."""
    if opts is None:
        opts = B.make_opts(**kw)
    Bb = [op._batch(b, op.k) for op, b in zip(ops, Bs)]
    Xs = [b.new_empty(b.shape) for b in Bb]   # zeroed by the library (no start given)
    opts.use_x0 = 0
    allow = (B.SYLV_E_NOT_CONVERGED,) if allow_not_converged else ()
    code, infos = B.sylv_solve_batched([op.handle for op in ops], Bb, Xs,
                                       [b.shape[0] for b in Bb], opts,
                                       shapes=[(op.k, op.ld, op.n) for op in ops],
                                       stream=stream, allow=allow)
    return Xs, [i.as_dict() for i in infos]
