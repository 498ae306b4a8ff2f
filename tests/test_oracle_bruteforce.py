"""Oracle forward pinned by brute force.

* Fanout-free circuits with up to 20 startpoints: input independence holds at every gate,
  so the propagated SP (Algorithm 2) must equal the exact probability obtained by enumerating
  all 2^n input assignments (weighted by their probabilities).
* Any circuit with 0/1 inputs: SP equals the Boolean value of every net (wiring pin).
* Reconvergent fanout breaks independence: the propagated SP differs from the truth there;
  this documents the model's known error (Sec. II-B), not a defect.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests import _gates as G


def random_tree(rng, n_inputs):
    """Fanout-free circuit: every net feeds at most one cell. Returns netlist text."""
    lines, free, nid, cid = [], [], 0, 0
    for i in range(n_inputs):
        lines.append(f"net n{nid} {rng.uniform(0.5, 2):.4f}")
        lines.append(f"input n{nid}")
        free.append(nid)
        nid += 1
    while len(free) > 1:
        gate = G.NAMES[rng.integers(len(G.NAMES))]
        ins, out, _ = G.BOOL[gate]
        if len(ins) > len(free):
            continue
        pick = [free.pop(rng.integers(len(free))) for _ in ins]
        lines.append(f"net n{nid} {rng.uniform(0.5, 2):.4f}")
        drv = ["X1", "X2", "X4"][rng.integers(3)]
        lines.append(f"cell u{cid} {gate}_{drv} " + " ".join(f"{p}=n{x}" for p, x in zip(ins, pick)) + f" {out}=n{nid}")
        free.append(nid)
        nid += 1
        cid += 1
    # a few single-input cells on top for depth
    for _ in range(3):
        gate = ["INV", "BUF"][rng.integers(2)]
        ins, out, _ = G.BOOL[gate]
        x = free.pop()
        lines.append(f"net n{nid} 1.0")
        lines.append(f"cell u{cid} {gate}_X1 {ins[0]}=n{x} {out}=n{nid}")
        free.append(nid)
        nid += 1
        cid += 1
    return "\n".join(lines) + "\n"


def exact_sp(text, p):
    """P(net = 1) for every net by enumeration of all 2^n startpoint assignments."""
    n = len(p)
    m = np.arange(2 ** n, dtype=np.int64)
    bits = ((m[None, :] >> np.arange(n)[:, None]) & 1).astype(np.int64)     # [n, 2^n]
    w = np.prod(np.where(bits == 1, p[:, None], 1 - p[:, None]), axis=0)     # [2^n]
    vals = G.boolean_eval(text, list(bits))                                   # [nets, 2^n]
    return (vals * w[None, :]).sum(axis=1)


@pytest.mark.parametrize("seed,n", [(1, 2), (2, 5), (3, 9), (4, 14), (5, 17), (6, 20)])
def test_fanout_free_equals_enumeration(seed, n, library_text):
    rng = np.random.default_rng(seed)
    text = random_tree(rng, n)
    o = Oracle(text, library_text)
    p = rng.uniform(0.05, 0.95, n)
    sp, tr = o.forward(p, np.zeros(n))
    want = exact_sp(text, p)
    np.testing.assert_allclose(sp, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["small", "mid"])
def test_boolean_inputs_give_boolean_values(name, library_text):
    spec = netgen.WORKLOADS[name]
    text = netgen.netlist_text(spec)
    o = Oracle(text, library_text)
    rng = np.random.default_rng(3)
    for _ in range(3):
        bits = rng.integers(0, 2, o.n_start)
        sp, tr = o.forward(bits.astype(float), np.zeros(o.n_start))
        want = G.boolean_eval(text, list(bits.astype(np.int64)))
        np.testing.assert_array_equal(sp, want.astype(float))
        cells = o.cell_outs()
        np.testing.assert_array_equal(tr[cells], 0.0)


def test_reconvergence_is_the_models_error(library_text):
    # y = XOR(BUF(a), BUF(a)) is constant 0, but the independence model gives 2p(1-p)
    text = ("net a 1\nnet b 1\nnet c 1\nnet y 1\ninput a\n"
            "cell u1 BUF_X1 A=a Z=b\ncell u2 BUF_X1 A=a Z=c\ncell u3 XOR2_X1 A=b B=c Z=y\n")
    o = Oracle(text, library_text)
    sp, _ = o.forward(np.array([0.3]), np.zeros(1))
    assert exact_sp(text, np.array([0.3]))[3] == 0.0
    assert sp[3] == pytest.approx(2 * 0.3 * 0.7, abs=1e-15)


def test_generator_structure(library_text):
    # the generated netlist has the requested sizes and exact depth
    for name in ["small", "mid"]:
        spec = netgen.WORKLOADS[name]
        o = Oracle(netgen.netlist_text(spec), library_text)
        assert o.n_cells == spec.n_cells and o.n_start == spec.n_start and o.depth == spec.depth
        assert o.n_nets == spec.n_cells + spec.n_start
