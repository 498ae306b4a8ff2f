"""PyTorch face of the library: a resident design, the model power as a
``torch.autograd.Function``, and the gradient-ascent power-virus search of
Algorithm 4 driven through it.

Argument marshalling only: every arithmetic step runs in the library's CUDA
kernels (``dp.*`` calls on raw device pointers).  PyTorch supplies device
memory, streams, CUDA-graph capture and the autograd bookkeeping.

Layouts follow the C-ABI: per-startpoint inputs are ``[n_start, S]`` float32
(scenario innermost), powers ``[S]`` float64, cap gradients ``[n_cells]``.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import dp


class Design:
    """A compiled netlist resident on one GPU, with the context whose stream the
    library follows (each call switches it to PyTorch's current stream)."""

    def __init__(self, netlist: str, library: str, device: int = 0):
        self.device = torch.device("cuda", device)
        self.ctx = dp.dp_create(device, torch.cuda.current_stream(self.device).cuda_stream)
        try:
            self.d = dp.dp_design_load(self.ctx, netlist, library)
        except Exception:
            dp.dp_destroy(self.ctx)
            raise
        info = dp.dp_design_info(self.d)
        self.n_start, self.n_cells, self.n_nets = info.n_start, info.n_cells, info.n_nets
        self.version = 0      # bumped by every forward; a stale backward recomputes its forward

    def follow_stream(self) -> None:
        dp.dp_set_stream(self.ctx, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self) -> None:
        if getattr(self, "d", None):
            dp.dp_design_free(self.d)
            self.d = None
        if getattr(self, "ctx", None):
            dp.dp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_input(x: torch.Tensor, rows: int, name: str) -> int:
    if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.shape[0] == rows
            and x.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape [{rows}, S]")
    return int(x.shape[1])


def _forward(design: Design, cfg, sp: torch.Tensor, tr: torch.Tensor, pincap, out: torch.Tensor) -> None:
    design.follow_stream()
    if pincap is not None:
        dp.dp_set_pincap_all(design.ctx, design.d, pincap, design.n_cells, on_device=1)
    dp.dp_set_inputs_batch(design.ctx, design.d, sp, tr, int(sp.shape[1]), on_device=1)
    dp.dp_propagate(design.ctx, design.d, cfg)
    dp.dp_get_power(design.ctx, design.d, out, 0, on_device=1)
    design.version += 1


class DiffPowerFunction(torch.autograd.Function):
    """P_s = K sum_n TR_n(s) C_n for every scenario s (Eq. 1, Eq. 2, Algorithm 2).

    forward(sp [n_start, S], tr [n_start, S], pincap [n_cells] or None, design, cfg) -> [S] float64
    backward: the weighted reverse pass (Sec. III-E, Eq. 7) with grad_output as the
    per-scenario weights; pin-cap gradients are summed over the scenarios in FP64.
    """

    @staticmethod
    def forward(ctx, sp, tr, pincap, design: Design, cfg):
        S = _check_input(sp, design.n_start, "sp")
        if _check_input(tr, design.n_start, "tr") != S:
            raise ValueError("sp and tr need the same number of scenarios")
        if pincap is not None and not (pincap.is_cuda and pincap.dtype == torch.float32
                                       and pincap.numel() == design.n_cells and pincap.is_contiguous()):
            raise ValueError("pincap must be a contiguous float32 CUDA tensor of n_cells values")
        out = torch.empty(S, dtype=torch.float64, device=sp.device)
        _forward(design, cfg, sp, tr, pincap, out)
        ctx.design, ctx.cfg, ctx.version = design, cfg, design.version
        ctx.has_pincap = pincap is not None
        ctx.save_for_backward(sp, tr, pincap if pincap is not None else sp.new_empty(0))
        return out

    @staticmethod
    def backward(ctx, grad_out):
        design, cfg = ctx.design, ctx.cfg
        sp, tr, pincap = ctx.saved_tensors
        if design.version != ctx.version:   # another forward ran since: restore this one's state
            scratch = torch.empty(sp.shape[1], dtype=torch.float64, device=sp.device)
            _forward(design, cfg, sp, tr, pincap if ctx.has_pincap else None, scratch)
            ctx.version = design.version
        design.follow_stream()
        w = grad_out if grad_out.is_contiguous() else grad_out.contiguous()
        if w.dtype != torch.float64:
            raise TypeError("the power gradient must be float64")
        need_sp, need_tr, need_pin = ctx.needs_input_grad[:3]
        gsp = torch.empty_like(sp) if need_sp else None
        gtr = torch.empty_like(tr) if need_tr else None
        gpin = torch.empty(design.n_cells, dtype=torch.float32, device=sp.device) if need_pin else None
        dp.dp_backward_weighted(design.ctx, design.d, cfg, w, 1, gsp, gtr, gpin, None, on_device=1)
        return gsp, gtr, gpin, None, None


def power(design: Design, sp: torch.Tensor, tr: torch.Tensor, pincap: torch.Tensor | None = None, *,
          tr_mode: int = 0, vdd: float = 0.8, fclk: float = 1e9) -> torch.Tensor:
    """Model power per scenario, differentiable in sp, tr and pincap."""
    cfg = dp.config(tr_mode=tr_mode, grad_mode=0, vdd=vdd, fclk=fclk)
    return DiffPowerFunction.apply(sp, tr, pincap, design, cfg)


@dataclass
class VirusResult:
    sp: torch.Tensor          # [n_start, S] final SP of every start
    tr: torch.Tensor          # [n_start, S] final TR
    v0: torch.Tensor          # [n_start, S] uint8 thresholded vector (v1 = 1 - v0)
    p_virus: torch.Tensor     # [S] float64, fF (Eq. 3)
    proxy_start: torch.Tensor # [S] float64, fF: sum C TR at the start
    proxy_end: torch.Tensor   # [S] float64, fF: at the end
    ms_ascent: float          # device time of the ascent steps (the replays, with a graph)
    graph: bool


def power_virus(design: Design, sp0: torch.Tensor, tr0: torch.Tensor, steps: int, eta_sp: float,
                eta_tr: float = 0.0, *, tr_mode: int = 1, vdd: float = 0.8, fclk: float = 1e9,
                graph: bool = True, warmup: int = 2) -> VirusResult:
    """Algorithm 4 for every start (scenario) at once.

    Each step differentiates the proxy sum_n C_n TR_n (the power divided by
    K = 1/2 Vdd^2 f; Eq. 9 in tr_mode 1) through :class:`DiffPowerFunction`
    and moves SP (and TR in tr_mode 0) by eta times its gradient, projected
    onto [0, 1].  With ``graph`` the step - forward, backward and update - is
    captured once in a CUDA graph (after ``warmup`` eager steps whose effect on
    the inputs is undone) and replayed ``steps`` times.  Then the final SP is thresholded (v0 = [SP >= 0.5], v1 = not v0)
    and P_virus (Eq. 3) is evaluated by two bitwise forward passes.
    """
    if steps < 0:
        raise ValueError("steps must be non-negative")
    cfg = dp.config(tr_mode=tr_mode, grad_mode=0, vdd=vdd, fclk=fclk)
    K = 0.5 * vdd * vdd * fclk * 1e-15
    S = _check_input(sp0, design.n_start, "sp0")
    x = sp0.detach().clone().requires_grad_(True)
    t = tr0.detach().clone().requires_grad_(tr_mode == 0)
    w = torch.full((S,), 1.0 / K, dtype=torch.float64, device=sp0.device)
    n = x.numel()

    def proxy() -> torch.Tensor:
        with torch.no_grad():
            return DiffPowerFunction.apply(x.detach(), t.detach(), None, design, cfg) / K

    def step() -> None:
        x.grad = None
        t.grad = None
        p = DiffPowerFunction.apply(x, t, None, design, cfg)
        p.backward(w)
        design.follow_stream()
        dp.dp_ascent_step(design.ctx, x, x.grad, n, eta_sp)
        if tr_mode == 0:
            dp.dp_ascent_step(design.ctx, t, t.grad, n, eta_tr)

    p_start = proxy()
    use_graph = graph and steps > 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if use_graph:
        # warm-up steps on the side stream (first-use allocations, autograd state), then the
        # starting point restored: all `steps` steps are replays of the captured step, and
        # the timing holds their device time alone
        with torch.no_grad():
            x0, t0 = x.detach().clone(), t.detach().clone()
        side = torch.cuda.Stream(sp0.device)
        side.wait_stream(torch.cuda.current_stream(sp0.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                step()
        torch.cuda.current_stream(sp0.device).wait_stream(side)
        with torch.no_grad():
            x.copy_(x0)
            t.copy_(t0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        ev0.record()
        for _ in range(steps):
            g.replay()
        ev1.record()
    else:
        ev0.record()
        for _ in range(steps):
            step()
        ev1.record()
    torch.cuda.synchronize(sp0.device)
    ms = ev0.elapsed_time(ev1)
    p_end = proxy()
    design.follow_stream()
    v0 = torch.empty_like(x, dtype=torch.uint8)
    pv = torch.empty(S, dtype=torch.float64, device=sp0.device)
    dp.dp_virus_eval(design.ctx, design.d, x.detach(), S, pv, v0, on_device=1)
    torch.cuda.synchronize(sp0.device)
    return VirusResult(x.detach(), t.detach(), v0, pv, p_start, p_end, ms, use_graph)
