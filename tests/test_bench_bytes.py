"""The compulsory-byte counts behind the benchmark's roofline fractions (no GPU): one forward +
reverse pass on the 2,000,000-cell netlist moves 54.8 + 89.2 = 144.0 MB (every structure or value
array read or written once, int32 indices, binary32 values), i.e. about 72 bytes per cell, and the
120,000-cell netlist's 4,096-vector simulation about 135 MB (every net's 512 bytes of words
written and read once)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sizes(nc, ns):
    # expected fanin edges: mean arity over the 13 generator functions is 29 / 13
    return nc + ns, ns, nc, round(nc * 29 / 13)


def test_fwd_bwd_compulsory_bytes():
    nn, ns, nc, ne = sizes(2_000_000, 147_456)
    b = bench.fwd_bwd_bytes(nn, ns, nc, ne)
    assert round(b["forward"] / 1e6, 1) == 54.8
    assert round(b["backward"] / 1e6, 1) == 89.2
    assert round(b["total"] / 1e6, 1) == 144.0
    assert 71 < b["total"] / nc < 73
    # by hand: forward = fanin CSR + startpoint SP/TR in + C_load in + SP/TR out
    fanin = 4 * (nc + 1) + 4 * ne + nc
    assert b["forward"] == fanin + 8 * ns + 4 * nn + 8 * nn
    # reverse = fanin CSR + SP + C_load + fanout CSR + adjoint out + pin-cap and startpoint gradients
    assert b["backward"] == fanin + 4 * nn + 4 * nn + 4 * (nn + 1) + 4 * ne + 4 * nn + 4 * nc + 8 * ns


def test_simulation_bytes():
    nn, ns, nc, ne = sizes(120_000, 9_216)
    assert 134e6 < bench.sim_bytes(nn, ns, nc, ne, 64) < 136e6
    assert bench.sim_bytes(nn, ns, nc, ne, 64) == 2 * 8 * 64 * nn + 4 * (nc + 1) + 4 * ne + nc + 8 * nn


def test_traffic_needs_the_captured_source():
    # reported only for the workload it was captured on (the source hash is checked as well)
    assert bench.kernel_traffic("k_sim_wide", "mid") is None
    assert bench.kernel_traffic("no_such_kernel", "roofline") is None
