"""Seeded synthetic inputs: netlists, the cell library and input-activity scenarios.

The paper's designs are proprietary or not shipped (Sec. V-A), so seeded random
netlists with the same structure stand in for them (recipe in ``gen/netgen.c``).
This module only draws structure, capacitances and input activities; it holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle may
use it.

Named workloads (cells, primary inputs, DFFs, depth, fanout cap, seed):

* ``small``    2,000 cells, 64 PIs + 32 DFFs, depth 24, cap 16, seed 1
* ``mid``      120,000 cells, 1,024 PIs + 8,192 DFFs, depth 48, cap 16, seed 2
* ``roofline`` 2,000,000 cells, 16,384 PIs + 131,072 DFFs, depth 80, cap 32, seed 3
* ``serve_<n>`` eight serving designs (5K ... 2M cells, seeds 1-8), startpoints
  and depth scaled from the three above.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen", "netgen.c")
_OUT = os.path.join(_HERE, "_out")
_SO = os.path.join(_OUT, "libnetgen.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_cells", ctypes.c_int64),
        ("n_pi", ctypes.c_int64),
        ("n_dff", ctypes.c_int64),
        ("depth", ctypes.c_int32),
        ("fanout_cap", ctypes.c_int32),
        ("p_prev", ctypes.c_double),
        ("shuffle", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compiles the generator into a shared library (plain C, any host arch)."""
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.ng_generate.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_int64)]
            lib.ng_generate.restype = ctypes.c_int
            lib.ng_library_text.argtypes = []
            lib.ng_library_text.restype = ctypes.c_void_p
            lib.ng_free.argtypes = [ctypes.c_void_p]
            lib.ng_free.restype = None
            _lib = lib
    return _lib


@dataclass(frozen=True)
class NetlistSpec:
    n_cells: int
    n_pi: int
    n_dff: int
    depth: int
    fanout_cap: int = 16
    seed: int = 1
    p_prev: float = 0.8
    shuffle: bool = True

    @property
    def n_start(self) -> int:
        return self.n_pi + self.n_dff


def _serve_spec(n_cells: int, seed: int) -> NetlistSpec:
    # startpoints ~7.4% of cells and depth growing with log size, as in the three named designs
    n_start = max(16, int(round(n_cells * 0.0737)))
    n_pi = max(8, n_start // 9)
    depth = int(min(80, max(16, round(24 + 14 * np.log10(n_cells / 2000.0)))))
    return NetlistSpec(n_cells, n_pi, n_start - n_pi, depth, 32 if n_cells >= 1_000_000 else 16, seed)


WORKLOADS = {
    "small": NetlistSpec(2_000, 64, 32, 24, 16, 1),
    "mid": NetlistSpec(120_000, 1_024, 8_192, 48, 16, 2),
    "roofline": NetlistSpec(2_000_000, 16_384, 131_072, 80, 32, 3),
}
for _i, _n in enumerate([5_000, 20_000, 50_000, 120_000, 300_000, 600_000, 1_000_000, 2_000_000]):
    WORKLOADS[f"serve_{_n}"] = _serve_spec(_n, _i + 1)


def _paper_spec(n_cells: int, depth: int, seed: int) -> NetlistSpec:
    # the cell count and depth of the paper's three designs (Table II / III); startpoints
    # as in the serving designs
    n_start = int(round(n_cells * 0.0737))
    n_pi = n_start // 9
    return NetlistSpec(n_cells, n_pi, n_start - n_pi, depth, 32 if n_cells >= 500_000 else 16, seed)


WORKLOADS["paper_small"] = _paper_spec(13_000, 70, 11)
WORKLOADS["paper_medium"] = _paper_spec(117_000, 84, 12)
WORKLOADS["paper_large"] = _paper_spec(652_000, 104, 13)


def library_text() -> str:
    """The synthetic library: 13 functions x X1/X2/X4 (pin cap 0.8/1.6/3.2 fF) and DFF_X1."""
    lib = _load()
    p = lib.ng_library_text()
    if not p:
        raise MemoryError("library text")
    try:
        return ctypes.string_at(p).decode()
    finally:
        lib.ng_free(p)


def netlist_text(spec: NetlistSpec) -> str:
    """Netlist text for ``spec`` (deterministic in ``spec.seed``)."""
    lib = _load()
    prm = _Params(spec.seed, spec.n_cells, spec.n_pi, spec.n_dff, spec.depth, spec.fanout_cap,
                  spec.p_prev, 1 if spec.shuffle else 0)
    out = ctypes.c_void_p()
    nn = ctypes.c_int64()
    rc = lib.ng_generate(ctypes.byref(prm), ctypes.byref(out), ctypes.byref(nn))
    if rc != 0:
        raise ValueError(f"netlist generator failed ({rc}) for {spec}")
    try:
        return ctypes.string_at(out).decode()
    finally:
        lib.ng_free(out)


def scenario_inputs(n_start: int, seed: int, n_scen: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Input SP ~ U[0.1, 0.9] and TR ~ U[0, 2 min(SP, 1-SP)] per startpoint, binary32.

    Returns arrays of shape ``[n_start, n_scen]`` (scenario innermost); scenario ``s``
    is drawn from seed ``seed + s``.
    """
    sp = np.empty((n_start, n_scen), np.float32)
    tr = np.empty((n_start, n_scen), np.float32)
    for s in range(n_scen):
        g = np.random.Generator(np.random.PCG64(seed + s))
        a = g.uniform(0.1, 0.9, n_start).astype(np.float32)
        hi = 2.0 * np.minimum(a.astype(np.float64), 1.0 - a.astype(np.float64))
        b = (g.uniform(0.0, 1.0, n_start) * hi).astype(np.float32)
        sp[:, s] = a
        tr[:, s] = np.minimum(b, hi.astype(np.float32))
    return sp, tr
