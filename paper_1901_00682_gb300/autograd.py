"""Differentiable unrolled solver: u_N = Phi_N(f, alpha) as a torch.autograd.Function.

Phi_N is N outer iterations of Algorithm 1 from the initial state of a load (u^0 = f,
p~ = 0, lambda = 0), computed by the CUDA library.  The backward pass is the
library's hand-written reverse pass (dd_tv_adjoint_backward): it recomputes each
segment of ``checkpoint_every`` outer iterations from a checkpoint kept by the
forward pass and runs the adjoint of every outer iteration of the segment in reverse
order, giving dL/df and dL/dalpha for the incoming dL/du_N.

Every image of a batch has its own library handle and CUDA stream; the images'
forward and backward passes are issued from a small thread pool (the ctypes calls
release the GIL), so they run concurrently on the GPU.  A handle keeps the
checkpoints of one forward pass, so every forward whose backward may still come gets
its own set of handles: a set is lent to a forward until the autograd graph that holds
that forward is freed (then it is reused), so several forwards may run before their
backwards.  Argument marshalling only: all arithmetic runs in the library.
"""
from __future__ import annotations

import weakref
from concurrent.futures import ThreadPoolExecutor

import torch

from . import _lib as L


class UnrolledDDTV:
    """Callable u = m(f, alpha, mask=None) with f of shape (B, H, W) or (H, W)
    (float32, CUDA, contiguous) and alpha a float, a 0-d tensor (shared by the batch)
    or a (B,) tensor.  Gradients flow to f and to alpha when they require them."""

    def __init__(self, height, width, sub_rows, sub_cols, n_outer, checkpoint_every=10, fidelity="l2", c1=0.0,
                 c2=0.0, inner_iters=10, path="fused", variant=0, **steps):
        self.shape = (height, width)
        self.n_outer = int(n_outer)
        self.every = int(checkpoint_every)
        self.kw = dict(sub_rows=sub_rows, sub_cols=sub_cols, fidelity=fidelity, c1=c1, c2=c2,
                       inner_iters=inner_iters, path=path, variant=variant, **steps)
        self._sets = []      # handle sets: {"handles": [(Solver, torch.cuda.Stream)], "owner": weakref | None}
        self._pool = None

    def _lend(self, n, alpha0, ctx):
        """A handle set of at least n handles whose checkpoints no live forward needs,
        lent to ctx (the forward's autograd context) until ctx is freed."""
        free = None
        for hs in self._sets:
            if hs["owner"] is None or hs["owner"]() is None:
                free = hs
                break
        if free is None:
            free = {"handles": [], "owner": None}
            self._sets.append(free)
        while len(free["handles"]) < n:
            st = torch.cuda.Stream()
            p = L.make_params(*self.shape, alpha=alpha0, outer_iters=self.n_outer, **self.kw)
            free["handles"].append((L.Solver(p, st), st))
        free["owner"] = weakref.ref(ctx)
        if self._pool is None or self._pool._max_workers < n:
            if self._pool is not None:
                self._pool.shutdown()
            self._pool = ThreadPoolExecutor(max_workers=n)
        return free

    def close(self):
        for hs in self._sets:
            for s, _ in hs["handles"]:
                s.close()
        self._sets = []
        if self._pool is not None:
            self._pool.shutdown()
            self._pool = None

    def __call__(self, f, alpha, mask=None):
        squeeze = f.dim() == 2
        if squeeze:
            f = f.unsqueeze(0)
            mask = None if mask is None else mask.unsqueeze(0)
        if not isinstance(alpha, torch.Tensor):
            alpha = torch.tensor(float(alpha), dtype=torch.float64, device=f.device)
        u = _UnrolledFn.apply(f, alpha, mask, self)
        return u.squeeze(0) if squeeze else u


class _UnrolledFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, alpha, mask, mod):
        if f.dtype != torch.float32 or not f.is_cuda:
            raise TypeError("f must be a float32 CUDA tensor")
        f = f.contiguous()
        B = f.shape[0]
        al = alpha.detach().reshape(-1).double().cpu().tolist()
        if len(al) not in (1, B):
            raise ValueError("alpha must be a scalar or have one entry per image")
        al = al * B if len(al) == 1 else al
        lent = mod._lend(B, al[0], ctx)
        hs = lent["handles"][:B]
        m = None if mask is None else mask.to(torch.uint8).contiguous()
        u = torch.empty_like(f)
        cur = torch.cuda.current_stream()
        for _, st in hs:
            st.wait_stream(cur)

        fb, ub = list(f.unbind(0)), list(u.unbind(0))
        mb = [None] * B if m is None else list(m.unbind(0))

        def fwd(b):
            s, _ = hs[b]
            if s.params.alpha != al[b]:
                s.set_alpha(al[b])
            s.adjoint_forward(fb[b], mb[b], mod.n_outer, mod.every, ub[b])

        list(mod._pool.map(fwd, range(B)))
        for _, st in hs:
            cur.wait_stream(st)
        ctx.mod, ctx.B, ctx.alpha_shape, ctx.lent = mod, B, alpha.shape, lent
        ctx.alpha_dtype = alpha.dtype
        return u

    @staticmethod
    def backward(ctx, gu):
        mod, B = ctx.mod, ctx.B
        hs = ctx.lent["handles"][:B]
        gu = gu.contiguous().float()
        gf = torch.empty_like(gu)
        cur = torch.cuda.current_stream()
        for _, st in hs:
            st.wait_stream(cur)
        gub, gfb = list(gu.unbind(0)), list(gf.unbind(0))
        ga = list(mod._pool.map(lambda b: hs[b][0].adjoint_backward(gub[b], gfb[b]), range(B)))
        for _, st in hs:
            cur.wait_stream(st)
        g_alpha = None
        if ctx.needs_input_grad[1]:
            t = torch.tensor(ga, dtype=torch.float64)
            t = t.sum() if len(ctx.alpha_shape) == 0 or ctx.alpha_shape.numel() == 1 else t
            g_alpha = t.reshape(ctx.alpha_shape).to(dtype=ctx.alpha_dtype, device=gu.device)
        return (gf if ctx.needs_input_grad[0] else None), g_alpha, None, None


if __name__ == "__main__":
    # Forward + backward of the unrolled solver on synthetic ROF images (the
    # differentiation workload's recipe) and their wall times:
    #   python -m paper_1901_00682_gb300.autograd [images] [side] [outer] [checkpoint_every]
    import sys
    import time

    import numpy as np

    import synth
    args = [int(x) for x in sys.argv[1:]]
    B, S, N, M = (args + [8, 1024, 100, 10][len(args):])[:4]
    pairs = [synth.rof_image(S, S, max(4, 400 * S * S // (4096 * 4096)), 0.08, 500 + b) for b in range(B)]
    f = torch.from_numpy(np.stack([p[0] for p in pairs])).cuda().requires_grad_(True)
    g = torch.from_numpy(np.stack([p[1] for p in pairs])).cuda()
    alpha = torch.tensor(10.0, dtype=torch.float64, device="cuda", requires_grad=True)
    mod = UnrolledDDTV(S, S, S // 128, S // 128, N, checkpoint_every=M)
    for rep in range(2):
        f.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = mod(f, alpha)
        loss = 0.5 * ((u - g) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    print(f"{B} x {S}^2, {N} outer: forward {1e3 * (t1 - t0):.2f} ms, backward {1e3 * (t2 - t1):.2f} ms, "
          f"loss {loss.item():.6e}, dL/dalpha {alpha.grad.item():.6e}")
    mod.close()
