"""Python handle on the FP64 CPU oracle (``dpo.c``).  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the GPU package and the
GPU package never imports it.  Inputs are netlist/library text and numpy
arrays; all outputs are numpy arrays in the netlist's own order (nets in
declaration order, startpoints in order of appearance, cells in order of
appearance).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpo.c")
_OUT = os.path.join(_HERE, "_out")
_SO = os.path.join(_OUT, "liboracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_F = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compiles the oracle with the host C compiler (no GPU code)."""
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP only for the level-parallel baseline; without it those functions run serially
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _opt(ptr_type):
    """ndpointer that also accepts None."""
    class _Opt(ptr_type):  # type: ignore[misc, valid-type]
        @classmethod
        def from_param(cls, obj):
            return None if obj is None else ptr_type.from_param(obj)
    return _Opt


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_load.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]
            L.orc_load.restype = _P
            L.orc_free.argtypes = [_P]
            L.orc_info.argtypes = [_P, _I64]
            L.orc_start_nets.argtypes = [_P, _I64]
            L.orc_cell_outs.argtypes = [_P, _I64]
            L.orc_set_pincap.argtypes = [_P, ctypes.c_int64, ctypes.c_double]
            L.orc_cload.argtypes = [_P, _D]
            L.orc_forward.argtypes = [_P, _D, _D, ctypes.c_int, _D, _D, _D]
            L.orc_forward.restype = ctypes.c_int
            L.orc_power.argtypes = [_P, _D, ctypes.c_double, ctypes.c_double]
            L.orc_power.restype = ctypes.c_double
            L.orc_backward.argtypes = [_P, _D, _D, _opt(_D), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _opt(_D), _opt(_D), _opt(_D), _opt(_D), _opt(_D)]
            L.orc_backward.restype = ctypes.c_int
            L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.orc_simulate.argtypes = [_P, _F, _F, ctypes.c_uint64, ctypes.c_int, _opt(_U64), _U32, _U32]
            L.orc_simulate.restype = ctypes.c_int
            L.orc_hybrid.argtypes = [_P, _D, _U32, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
            L.orc_logic_words.argtypes = [_P, _U64, _U64]
            L.orc_forward_lag1.argtypes = [_P, _D, _D, _D, _D, _D]
            L.orc_forward_lag1.restype = ctypes.c_int
            L.orc_backward_lag1.argtypes = [_P, _D, _D, ctypes.c_double, ctypes.c_double, _opt(_D), _opt(_D),
                                            _opt(_D), _opt(_D)]
            L.orc_backward_lag1.restype = ctypes.c_int
            L.orc_threads.restype = ctypes.c_int
            L.orc_forward_par.argtypes = L.orc_forward.argtypes
            L.orc_forward_par.restype = ctypes.c_int
            L.orc_backward_par.argtypes = L.orc_backward.argtypes
            L.orc_backward_par.restype = ctypes.c_int
            L.orc_simulate_par.argtypes = L.orc_simulate.argtypes
            L.orc_simulate_par.restype = ctypes.c_int
            _lib = L
    return _lib


def threads() -> int:
    """Host threads the level-parallel variants use (1 when built without OpenMP)."""
    return int(_load().orc_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: counter (4 x u32), key (2 x u32) -> 4 x u32."""
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32), out)
    return out


class Oracle:
    """FP64 reference for one netlist."""

    def __init__(self, netlist: str, library: str):
        L = _load()
        err = ctypes.create_string_buffer(512)
        h = L.orc_load(netlist.encode(), library.encode(), err, 512)
        if not h:
            raise ValueError(f"oracle: {err.value.decode()}")
        self._h = h
        info = np.zeros(5, np.int64)
        L.orc_info(h, info)
        self.n_nets, self.n_start, self.n_cells, self.n_edges, self.depth = (int(x) for x in info)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def start_nets(self) -> np.ndarray:
        out = np.zeros(self.n_start, np.int64)
        _load().orc_start_nets(self._h, out)
        return out

    def cell_outs(self) -> np.ndarray:
        out = np.zeros(self.n_cells, np.int64)
        _load().orc_cell_outs(self._h, out)
        return out

    def set_pincap(self, cell: int, cap: float) -> None:
        _load().orc_set_pincap(self._h, int(cell), float(cap))

    def cload(self) -> np.ndarray:
        out = np.zeros(self.n_nets, np.float64)
        _load().orc_cload(self._h, out)
        return out

    def forward(self, sp_in, tr_in, tr_mode: int = 0, want_sq: bool = False, parallel: bool = False):
        """Per-net SP and TR (Algorithm 2, Eq. 2) from startpoint inputs (binary32 inputs
        convert exactly; binary64 inputs allow finite differences).  With ``want_sq`` also
        P(net = 0), evaluated as its own probability sum rather than as 1 - SP."""
        sp = np.zeros(self.n_nets, np.float64)
        tr = np.zeros(self.n_nets, np.float64)
        sq = np.zeros(self.n_nets, np.float64)
        f = _load().orc_forward_par if parallel else _load().orc_forward
        f(self._h, np.ascontiguousarray(sp_in, np.float64), np.ascontiguousarray(tr_in, np.float64), int(tr_mode),
          sp, tr, sq)
        return (sp, tr, sq) if want_sq else (sp, tr)

    def power(self, alpha, vdd: float = 0.8, fclk: float = 1e9) -> float:
        """Eq. 1 in watts, caps in fF."""
        return float(_load().orc_power(self._h, np.ascontiguousarray(alpha, np.float64), vdd, fclk))

    def backward(self, sp_in, tr_in, beta=None, grad_mode: int = 0, tr_mode: int = 0,
                 vdd: float = 0.8, fclk: float = 1e9, parallel: bool = False) -> dict:
        """Gradients of Eq. 1 at the startpoint inputs (Eq. 7; Eq. 6 for grad_mode 1).  The
        hybrid modes (grad_mode 1, 2) differentiate sum K beta TR C with the given beta.
        ``parallel``: the level-parallel variant (each net gathers over its sinks)."""
        out = {
            "grad_sp_in": np.zeros(self.n_start), "grad_tr_in": np.zeros(self.n_start),
            "grad_pincap": np.zeros(self.n_cells), "grad_cload": np.zeros(self.n_nets),
            "grad_net": np.zeros(self.n_nets),
        }
        if grad_mode and beta is None:
            raise ValueError("beta required for hybrid gradient modes")
        f = _load().orc_backward_par if parallel else _load().orc_backward
        rc = f(self._h, np.ascontiguousarray(sp_in, np.float64),
                                  np.ascontiguousarray(tr_in, np.float64),
                                  None if beta is None else np.ascontiguousarray(beta, np.float64),
                                  int(grad_mode), int(tr_mode), vdd, fclk, out["grad_sp_in"],
                                  out["grad_tr_in"], out["grad_pincap"], out["grad_cload"], out["grad_net"])
        if rc != 0:
            raise MemoryError("oracle backward")
        return out

    def simulate(self, sp_in, tr_in, seed: int = 42, T: int = 64, want_words: bool = False,
                 parallel: bool = False):
        """Bit-packed Markov simulation: (toggles, ones[, words[n_nets, T]])."""
        tg = np.zeros(self.n_nets, np.uint32)
        on = np.zeros(self.n_nets, np.uint32)
        words = np.zeros((self.n_nets, T), np.uint64) if want_words else None
        f = _load().orc_simulate_par if parallel else _load().orc_simulate
        rc = f(self._h, np.ascontiguousarray(sp_in, np.float32),
                                  np.ascontiguousarray(tr_in, np.float32), int(seed), int(T), words, tg, on)
        if rc != 0:
            raise MemoryError("oracle simulate")
        return (tg, on, words) if want_words else (tg, on)

    def hybrid(self, tr_model, toggles, T: int = 64, beta_min: float = 0.1, beta_max: float = 10.0):
        """Eq. 4-5: (beta, hybrid TR) per net."""
        beta = np.zeros(self.n_nets)
        trh = np.zeros(self.n_nets)
        _load().orc_hybrid(self._h, np.ascontiguousarray(tr_model, np.float64),
                           np.ascontiguousarray(toggles, np.uint32), int(T), beta_min, beta_max, beta, trh)
        return beta, trh

    def step(self, sp_in, tr_in, *, seed: int = 42, T: int = 64, grad_mode: int = 1, tr_mode: int = 0,
             vdd: float = 0.8, fclk: float = 1e9, beta_min: float = 0.1, beta_max: float = 10.0,
             parallel: bool = False) -> dict:
        """The whole hot path once: forward, power, simulation, hybrid, adjoint (``parallel``:
        the level-parallel variants of the forward pass, simulation and adjoint)."""
        sp, tr = self.forward(sp_in, tr_in, tr_mode, parallel=parallel)
        p_model = self.power(tr, vdd, fclk)
        tg, on = self.simulate(sp_in, tr_in, seed, T, parallel=parallel)
        beta, trh = self.hybrid(tr, tg, T, beta_min, beta_max)
        p_hyb = self.power(trh, vdd, fclk)
        g = self.backward(sp_in, tr_in, beta if grad_mode else None, grad_mode, tr_mode, vdd, fclk,
                          parallel=parallel)
        g.update(sp=sp, tr=tr, toggles=tg, ones=on, beta=beta, tr_hyb=trh, power_model=p_model,
                 power_hybrid=p_hyb)
        return g

    # ---- batched scenarios, Algorithm 4 and Eq. 3 ----
    # A batch is S independent scenarios; arrays are [rows, S] (scenario innermost).

    def forward_batch(self, sp_in, tr_in, tr_mode: int = 0):
        """Per-net SP and TR [n_nets, S] of every scenario (each an independent forward pass)."""
        sp_in = np.asarray(sp_in)
        S = sp_in.shape[1]
        sp = np.zeros((self.n_nets, S))
        tr = np.zeros((self.n_nets, S))
        for s in range(S):
            sp[:, s], tr[:, s] = self.forward(sp_in[:, s], np.asarray(tr_in)[:, s], tr_mode)
        return sp, tr

    def backward_batch(self, sp_in, tr_in, weights=None, tr_mode: int = 0, vdd: float = 0.8,
                       fclk: float = 1e9) -> dict:
        """Model gradients (Eq. 7) of sum_s w_s P_s, per scenario ([rows, S]); the cap
        gradients also summed over the scenarios ("grad_pincap_sum", "grad_cload_sum")."""
        sp_in = np.asarray(sp_in)
        tr_in = np.asarray(tr_in)
        S = sp_in.shape[1]
        w = np.ones(S) if weights is None else np.asarray(weights, np.float64)
        out = {k: np.zeros((n, S)) for k, n in [("grad_sp_in", self.n_start), ("grad_tr_in", self.n_start),
                                                ("grad_pincap", self.n_cells), ("grad_cload", self.n_nets)]}
        for s in range(S):
            g = self.backward(sp_in[:, s], tr_in[:, s], None, 0, tr_mode, vdd, fclk)
            for k in out:
                out[k][:, s] = w[s] * g[k]
        out["grad_pincap_sum"] = out["grad_pincap"].sum(axis=1)
        out["grad_cload_sum"] = out["grad_cload"].sum(axis=1)
        return out

    def logic(self, start_words) -> np.ndarray:
        """Logic value words of every net (bit b = vector b) from startpoint words."""
        out = np.zeros(self.n_nets, np.uint64)
        _load().orc_logic_words(self._h, np.ascontiguousarray(start_words, np.uint64), out)
        return out

    def p_virus(self, sp_in):
        """Eq. 3 for candidate inputs sp_in [n_start, S] (Algorithm 4, last steps): v0 =
        [sp >= 0.5] decided in binary32, v1 = not v0, logic values of both vectors, and
        per scenario the exactly rounded sum of C_load (fF) over the nets that differ.
        Returns (p_virus[S], v0[n_start, S] as uint8)."""
        sp32 = np.asarray(sp_in, np.float32)
        S = sp32.shape[1]
        v0 = (sp32 >= np.float32(0.5)).astype(np.uint8)
        cl = self.cload()
        out = np.zeros(S)
        for s in range(S):
            # bit 0 carries v0, bit 1 carries v1 = not v0
            w = v0[:, s].astype(np.uint64) | ((1 - v0[:, s]).astype(np.uint64) << np.uint64(1))
            vals = self.logic(w)
            diff = ((vals ^ (vals >> np.uint64(1))) & np.uint64(1)).astype(bool)
            out[s] = math.fsum(cl[diff].tolist())
        return out, v0

    def ascent(self, sp_in, tr_in, steps: int, eta_sp: float, eta_tr: float = 0.0, tr_mode: int = 1,
               vdd: float = 0.8, fclk: float = 1e9):
        """Algorithm 4 on every scenario ([n_start, S]) in binary64: each step takes the gradient of
        the proxy sum_n C_n TR_n (the power divided by K = 1/2 Vdd^2 f; Eq. 9 when tr_mode is 1)
        at the current inputs, then SP <- clip(SP + eta_sp dSP, 0, 1) and, in tr_mode 0,
        TR <- clip(TR + eta_tr dTR, 0, 1).  Returns the final (sp, tr)."""
        K = 0.5 * vdd * vdd * fclk * 1e-15
        sp = np.array(sp_in, np.float64)
        tr = np.array(tr_in, np.float64)
        for _ in range(steps):
            for s in range(sp.shape[1]):
                g = self.backward(sp[:, s], tr[:, s], None, 0, tr_mode, vdd, fclk)
                sp[:, s] = np.clip(sp[:, s] + eta_sp * (g["grad_sp_in"] / K), 0.0, 1.0)
                if tr_mode == 0:
                    tr[:, s] = np.clip(tr[:, s] + eta_tr * (g["grad_tr_in"] / K), 0.0, 1.0)
        return sp, tr

    def proxy(self, sp_in, tr_in, tr_mode: int = 1) -> float:
        """sum_n C_n TR_n in fF (the power without K; Eq. 9 when tr_mode is 1)."""
        _, tr = self.forward(sp_in, tr_in, tr_mode)
        cl = self.cload()
        return math.fsum((tr * cl).tolist())

    # ---- lag-one mode ----

    def forward_lag1(self, sp_in, tr_in):
        """Per-net SP and lag-one TR: T_y = sum_(a,b) prod_i q_i(a_i, b_i) [f(a) != f(b)] with
        q(1,1) = P - T/2, q(0,0) = P(x=0) - T/2, q(0,1) = q(1,0) = T/2 (inputs must satisfy
        T <= 2 min(P, 1 - P))."""
        sp = np.zeros(self.n_nets)
        tr = np.zeros(self.n_nets)
        sq = np.zeros(self.n_nets)
        _load().orc_forward_lag1(self._h, np.ascontiguousarray(sp_in, np.float64),
                                 np.ascontiguousarray(tr_in, np.float64), sp, tr, sq)
        return sp, tr

    def backward_lag1(self, sp_in, tr_in, vdd: float = 0.8, fclk: float = 1e9) -> dict:
        """Gradients of K sum_n T_n C_n in the lag-one mode."""
        out = {"grad_sp_in": np.zeros(self.n_start), "grad_tr_in": np.zeros(self.n_start),
               "grad_pincap": np.zeros(self.n_cells), "grad_cload": np.zeros(self.n_nets)}
        rc = _load().orc_backward_lag1(self._h, np.ascontiguousarray(sp_in, np.float64),
                                       np.ascontiguousarray(tr_in, np.float64), vdd, fclk, out["grad_sp_in"],
                                       out["grad_tr_in"], out["grad_pincap"], out["grad_cload"])
        if rc != 0:
            raise MemoryError("oracle backward_lag1")
        return out

    # ---- sizing score (Eq. 8) ----

    def sizing_scores(self, sp_in, tr_in, mode: int = 0, tr_mode: int = 0, vdd: float = 0.8, fclk: float = 1e9,
                      eps: float = 1e-6):
        """Per cell line: S = |dP/dP_sw| * P_sw with P_sw = K TR C_load of the cell's output net.
        mode 0: dP/dP_sw read as the SP adjoint of the output net; mode 1: the chain rule through
        Eq. 2, adjoint / (2 - 4 SP), with |2 - 4 SP| floored at eps.  Returns (scores, p_sw)."""
        K = 0.5 * vdd * vdd * fclk * 1e-15
        sp, tr = self.forward(sp_in, tr_in, tr_mode)
        g = self.backward(sp_in, tr_in, None, 0, tr_mode, vdd, fclk)["grad_net"]
        cl = self.cload()
        y = self.cell_outs()
        psw = K * tr[y] * cl[y]
        if mode == 0:
            sens = np.abs(g[y])
        else:
            d = 2.0 - 4.0 * sp[y]
            d = np.where(np.abs(d) < eps, np.where(d < 0, -eps, eps), d)
            sens = np.abs(g[y] / d)
        return sens * psw, psw
