"""PyTorch front end: device tensors in, device tensors out, autograd through the CUDA adjoint.

Torch is used only to allocate outputs/workspace on the current device and to name the
current stream; the computation is the C library's.
"""
from __future__ import annotations

import torch

from .binding import (Formula, FormulaSet, StlParams, params as make_params, pipeline_staging_size,
                      robustness_and_backward_raw, robustness_backward_raw, robustness_host_pipelined_raw,
                      robustness_ragged_backward_raw, robustness_ragged_raw, robustness_raw)


def _check_sig(f: Formula, sig: torch.Tensor):
    if not sig.is_cuda:
        raise ValueError("signal must be a CUDA tensor (libstl has no CPU path)")
    if sig.dtype != torch.float32 or sig.dim() != 3 or sig.shape[2] != f.D:
        raise ValueError(f"signal must be float32 [B, T, {f.D}]")
    return sig.contiguous()


def _bounds(f: Formula, bounds, sig):
    if f.n_slots == 0:
        return None
    if bounds is None:
        raise ValueError("formula uses per-trace bounds; pass bounds [B, n_slots, 2]")
    b = bounds.to(device=sig.device, dtype=torch.float32).contiguous()
    if b.shape != (sig.shape[0], f.n_slots, 2):
        raise ValueError(f"bounds must be [B, {f.n_slots}, 2]")
    return b


def _ws(f, B, T, p, backward, device):
    n = f.workspace_size(B, T, p, backward)
    if n == 0:
        return None, 0
    return torch.empty(n // 4 + 1, dtype=torch.float32, device=device), n


def robustness(f: Formula, sig: torch.Tensor, bounds=None, p: StlParams | None = None) -> torch.Tensor:
    """Robustness trace [B, T] of formula ``f`` for signals ``sig`` [B, T, D] (no autograd)."""
    p = p or make_params()
    sig = _check_sig(f, sig)
    B, T, _ = sig.shape
    b = _bounds(f, bounds, sig)
    out = torch.empty((B, T), dtype=torch.float32, device=sig.device)
    ws, nws = _ws(f, B, T, p, False, sig.device)
    stream = torch.cuda.current_stream(sig.device).cuda_stream
    robustness_raw(f, sig.data_ptr(), B, T, None if b is None else b.data_ptr(), p, out.data_ptr(),
                   None if ws is None else ws.data_ptr(), nws, stream)
    return out


def robustness_backward(f: Formula, sig: torch.Tensor, grad_out: torch.Tensor, bounds=None,
                        p: StlParams | None = None):
    """(grad_sig [B,T,D], grad_bounds [B,n_slots,2] or None) of sum(grad_out * rho)."""
    p = p or make_params()
    sig = _check_sig(f, sig)
    B, T, D = sig.shape
    b = _bounds(f, bounds, sig)
    g = grad_out.to(device=sig.device, dtype=torch.float32).contiguous()
    gsig = torch.empty((B, T, D), dtype=torch.float32, device=sig.device)
    gb = torch.empty((B, f.n_slots, 2), dtype=torch.float32, device=sig.device) if f.n_slots else None
    ws, nws = _ws(f, B, T, p, True, sig.device)
    stream = torch.cuda.current_stream(sig.device).cuda_stream
    robustness_backward_raw(f, sig.data_ptr(), B, T, None if b is None else b.data_ptr(), p, g.data_ptr(),
                            gsig.data_ptr(), None if gb is None else gb.data_ptr(),
                            None if ws is None else ws.data_ptr(), nws, stream)
    return gsig, gb


def robustness_and_grad(f: Formula, sig: torch.Tensor, grad_out: torch.Tensor, bounds=None,
                        p: StlParams | None = None):
    """(rho [B,T], grad_sig [B,T,D], grad_bounds [B,n_slots,2] or None) in one launch
    (stl_robustness_and_backward): for an upstream gradient known before the forward values,
    e.g. a loss linear in rho."""
    p = p or make_params()
    sig = _check_sig(f, sig)
    B, T, D = sig.shape
    b = _bounds(f, bounds, sig)
    g = grad_out.to(device=sig.device, dtype=torch.float32).contiguous()
    rho = torch.empty((B, T), dtype=torch.float32, device=sig.device)
    gsig = torch.empty((B, T, D), dtype=torch.float32, device=sig.device)
    gb = torch.empty((B, f.n_slots, 2), dtype=torch.float32, device=sig.device) if f.n_slots else None
    ws, nws = _ws(f, B, T, p, True, sig.device)
    stream = torch.cuda.current_stream(sig.device).cuda_stream
    robustness_and_backward_raw(f, sig.data_ptr(), B, T, None if b is None else b.data_ptr(), p, g.data_ptr(),
                                rho.data_ptr(), gsig.data_ptr(), None if gb is None else gb.data_ptr(),
                                None if ws is None else ws.data_ptr(), nws, stream)
    return rho, gsig, gb


class HostPipeline:
    """Robustness (and its gradient) of traces held in page-locked host tensors, with the
    copies overlapped with the kernels (stl_robustness_host_pipelined): chunks of ``chunk``
    traces rotate over three streams.  The device staging area is allocated once."""

    def __init__(self, f: Formula, T: int, p: StlParams | None = None, chunk: int = 64, backward: bool = True,
                 device="cuda"):
        self.f, self.T, self.p, self.chunk = f, T, p or make_params(), chunk
        self.dev = torch.device(device)
        self.nbytes = pipeline_staging_size(f, chunk, T, self.p, backward)
        self.staging = torch.empty(self.nbytes // 4 + 1, dtype=torch.float32, device=self.dev)

    def __call__(self, sig, grad_out=None, bounds=None, out=None, grad_sig=None, grad_bounds=None):
        """sig [B, T, D], grad_out [B, T] (optional) and the outputs are pinned CPU tensors;
        returns (out, grad_sig, grad_bounds), filled once the current stream reaches the end."""
        B = sig.shape[0]
        ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
        robustness_host_pipelined_raw(self.f, sig.data_ptr(), B, self.T, ptr(bounds), self.p, ptr(grad_out), ptr(out),
                                      ptr(grad_sig), ptr(grad_bounds), self.chunk, self.staging.data_ptr(),
                                      self.nbytes, torch.cuda.current_stream(self.dev).cuda_stream)
        return out, grad_sig, grad_bounds


def autotune(f: Formula, sig: torch.Tensor, bounds=None, p: StlParams | None = None, backward=False,
             max_workspace_bytes: int = 1 << 30):
    """Tune the launch shape of ``f`` for this call shape (see stl_autotune); returns
    (launch, ms)."""
    p = p or make_params()
    sig = _check_sig(f, sig)
    B, T, D = sig.shape
    b = _bounds(f, bounds, sig)
    stream = torch.cuda.current_stream(sig.device).cuda_stream
    ws = torch.empty(max_workspace_bytes // 4, dtype=torch.float32, device=sig.device)
    if backward:
        # a dense upstream gradient: with zeros the smooth adjoints skip their work and the timing
        # would not be the real one
        g = torch.randn((B, T), dtype=torch.float32, device=sig.device)
        out = torch.empty((B, T, D), dtype=torch.float32, device=sig.device)
        gb = torch.empty((B, f.n_slots, 2), dtype=torch.float32, device=sig.device) if f.n_slots else None
        res = f.autotune(sig.data_ptr(), B, T, None if b is None else b.data_ptr(), p, True, g.data_ptr(),
                         out.data_ptr(), None if gb is None else gb.data_ptr(), ws.data_ptr(), ws.numel() * 4, stream)
    else:
        out = torch.empty((B, T), dtype=torch.float32, device=sig.device)
        res = f.autotune(sig.data_ptr(), B, T, None if b is None else b.data_ptr(), p, False, None, out.data_ptr(),
                         None, ws.data_ptr(), ws.numel() * 4, stream)
    del ws
    return res


class STLRobustness(torch.autograd.Function):
    """rho = STLRobustness.apply(formula, sig, bounds, params); differentiable w.r.t. sig and
    bounds.  The backward recomputes the forward on chip (no stored intermediates)."""

    @staticmethod
    def forward(ctx, f: Formula, sig, bounds, p):
        ctx.f, ctx.p = f, p
        ctx.save_for_backward(sig, bounds if bounds is not None else torch.empty(0, device=sig.device))
        ctx.has_bounds = bounds is not None
        return robustness(f, sig, bounds, p)

    @staticmethod
    def backward(ctx, grad_out):
        sig, bounds = ctx.saved_tensors
        gsig, gb = robustness_backward(ctx.f, sig, grad_out, bounds if ctx.has_bounds else None, ctx.p)
        return None, gsig, (gb if ctx.has_bounds else None), None


class RaggedBatch:
    """Device-resident ragged batch for a FormulaSet: packed signal [sum T, D], offsets, formula
    ids, optional processing order and bounds.  forward() / backward() each issue ONE launch and
    allocate nothing, so both can be captured in a CUDA graph (see capture())."""

    def __init__(self, fset: FormulaSet, sig, offsets, formula_id, bounds=None, p: StlParams | None = None,
                 order=None, device="cuda", tune=False):
        self.fset, self.p = fset, p or make_params()
        self.sig = sig.to(device=device, dtype=torch.float32).contiguous()
        self.offsets = offsets.to(device=device, dtype=torch.int64).contiguous()
        self.fid = formula_id.to(device=device, dtype=torch.int32).contiguous()
        self.order = None if order is None else order.to(device=device, dtype=torch.int32).contiguous()
        self.n = int(self.fid.numel())
        lens = (offsets[1:] - offsets[:-1])
        self.T_max = int(lens.max().item()) if self.n else 1
        self.bounds = None
        if fset.n_slots:
            if bounds is None:
                raise ValueError("the formulas use per-trace bounds")
            self.bounds = bounds.to(device=device, dtype=torch.float32).contiguous()
        total = int(offsets[-1].item())
        self.out = torch.empty(total, dtype=torch.float32, device=device)
        self.gsig = torch.empty((total, fset.D), dtype=torch.float32, device=device)
        self.gbounds = torch.empty((self.n, fset.n_slots, 2), device=device) if fset.n_slots else None
        self.shapes = None
        if tune and self.n:
            # stl_set_autotune per direction on this batch (a random upstream gradient for the
            # backward); the set is left prepared with the winners
            st = torch.cuda.current_stream(self.sig.device).cuda_stream
            g = torch.randn(total, device=device)
            args = (self.sig.data_ptr(), self.offsets.data_ptr(), self.fid.data_ptr(), self._ptr(self.order),
                    self._ptr(self.bounds))
            nf, shf, msf = fset.autotune(self.n, self.T_max, self.p, False, *args, None, self.out.data_ptr(), None, st)
            nb, shb, msb = fset.autotune(self.n, self.T_max, self.p, True, *args, g.data_ptr(), self.gsig.data_ptr(),
                                         self._ptr(self.gbounds), st)
            self.shapes = {"forward": {"threads": shf[0], "tile": shf[1], "ms": msf},
                           "backward": {"threads": shb[0], "tile": shb[1], "ms": msb}}
        else:
            nf = fset.prepare(max(1, self.n), self.T_max, self.p, False)
            nb = fset.prepare(max(1, self.n), self.T_max, self.p, True)
        self.ws_f = torch.empty(nf // 4 + 1, dtype=torch.float32, device=device)
        self.ws_b = torch.empty(nb // 4 + 1, dtype=torch.float32, device=device)
        self.nf, self.nb = nf, nb

    def _ptr(self, t):
        return None if t is None else t.data_ptr()

    def forward(self):
        st = torch.cuda.current_stream(self.sig.device).cuda_stream
        robustness_ragged_raw(self.fset, self.sig.data_ptr(), self.offsets.data_ptr(), self.fid.data_ptr(),
                              self._ptr(self.order), self.n, self._ptr(self.bounds), self.p, self.out.data_ptr(),
                              self.ws_f.data_ptr(), self.nf, st)
        return self.out

    def backward(self, grad_out):
        st = torch.cuda.current_stream(self.sig.device).cuda_stream
        robustness_ragged_backward_raw(self.fset, self.sig.data_ptr(), self.offsets.data_ptr(), self.fid.data_ptr(),
                                       self._ptr(self.order), self.n, self._ptr(self.bounds), self.p,
                                       grad_out.data_ptr(), self.gsig.data_ptr(), self._ptr(self.gbounds),
                                       self.ws_b.data_ptr(), self.nb, st)
        return self.gsig, self.gbounds

    def capture(self, grad_out):
        """Capture forward + backward into a CUDA graph (after one eager warm-up call)."""
        self.forward()
        self.backward(grad_out)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.forward()
                self.backward(grad_out)
        torch.cuda.current_stream().wait_stream(s)
        return g
