"""Oracle per-gate pins: closed-form SP and partials (Sec. III-E, the AND/OR/XOR/NOT rules),
Boolean truth tables of parsed expressions, and the parser's precedence NOT > AND > XOR > OR
(Sec. III-A)."""
import itertools

import numpy as np
import pytest

from oracle.oracle import Oracle
from tests import _gates as G

K = 0.5 * 0.8 ** 2 * 1e9 * 1e-15


def single_cell(gate, lib_text, wire_out=1.5):
    ins, out, _ = G.BOOL[gate]
    lines = [f"net i{j} 1.0" for j in range(len(ins))] + [f"net o {wire_out}"]
    lines += [f"input i{j}" for j in range(len(ins))]
    lines.append(f"cell u0 {gate}_X1 " + " ".join(f"{p}=i{j}" for j, p in enumerate(ins)) + f" {out}=o")
    return Oracle("\n".join(lines) + "\n", lib_text), len(ins)


@pytest.mark.parametrize("gate", G.NAMES)
def test_gate_sp_closed_form(gate, library_text):
    o, k = single_cell(gate, library_text)
    rng = np.random.default_rng(7)
    for _ in range(20):
        p = rng.uniform(0, 1, k)
        sp, tr = o.forward(p, np.zeros(k))
        want = G.SP[gate](*p)
        assert sp[k] == pytest.approx(want, abs=1e-15)
        assert tr[k] == pytest.approx(2 * want * (1 - want), abs=1e-15)


@pytest.mark.parametrize("gate", G.NAMES)
def test_gate_partials_closed_form(gate, library_text):
    # single gate: dP/dp_j = K C_out (2 - 4 sp_out) d sp_out / d p_j (startpoints have no local term)
    o, k = single_cell(gate, library_text, wire_out=1.5)
    rng = np.random.default_rng(11)
    for _ in range(20):
        p = rng.uniform(0.05, 0.95, k)
        g = o.backward(p, np.full(k, 0.1))
        s = G.SP[gate](*p)
        for j in range(k):
            want = K * 1.5 * (2 - 4 * s) * G.DSP[gate][j](*p)
            assert g["grad_sp_in"][j] == pytest.approx(want, rel=1e-12, abs=1e-22)


@pytest.mark.parametrize("gate", G.NAMES)
def test_gate_truth_table(gate, library_text):
    # with 0/1 inputs the SP is the Boolean value itself
    o, k = single_cell(gate, library_text)
    fn = G.BOOL[gate][2]
    for bits in itertools.product([0, 1], repeat=k):
        sp, _ = o.forward(np.array(bits, float), np.zeros(k))
        assert sp[k] == fn(*[np.int64(b) for b in bits])


PRECEDENCE = [
    ("A | B & C", lambda a, b, c: a | (b & c)),
    ("A & B | C", lambda a, b, c: (a & b) | c),
    ("A ^ B & C", lambda a, b, c: a ^ (b & c)),
    ("A | B ^ C", lambda a, b, c: a | (b ^ c)),
    ("!A & B | C", lambda a, b, c: ((1 - a) & b) | c),
    ("!(A | B) ^ C", lambda a, b, c: (1 - (a | b)) ^ c),
    ("A' * B + C", lambda a, b, c: ((1 - a) & b) | c),
    ("~A ^ ~B ^ C", lambda a, b, c: (1 - a) ^ (1 - b) ^ c),
    ("(A + B) * (B + C) & 1", lambda a, b, c: (a | b) & (b | c)),
    ("A & B & C | 0", lambda a, b, c: a & b & c),
]


@pytest.mark.parametrize("i", range(len(PRECEDENCE)))
def test_parser_precedence(i):
    expr, fn = PRECEDENCE[i]
    lib = f"cell F_X1 Y 1.0 {expr}\n"
    net = "net a 1\nnet b 1\nnet c 1\nnet y 1\ninput a\ninput b\ninput c\ncell u F_X1 A=a B=b C=c Y=y\n"
    o = Oracle(net, lib)
    for bits in itertools.product([0, 1], repeat=3):
        sp, _ = o.forward(np.array(bits, float), np.zeros(3))
        assert sp[3] == fn(*bits), (expr, bits)


@pytest.mark.parametrize("bad", [
    "net a 1\ninput a\ncell u NAND2_X1 A1=a A2=zz ZN=a\n",           # unknown net
    "net a 1\nnet b 1\ninput a\ncell u INV_X1 A=b ZN=b\n",             # cycle (self loop)
    "net a 1\nnet b 1\nnet c 1\ninput a\ncell u INV_X1 A=c ZN=b\ncell v INV_X1 A=b ZN=c\n",  # cycle
    "net a 1\nnet b 1\ninput a\ncell u NAND2_X1 A1=a ZN=b\n",          # missing pin
    "net a 1\nnet b 1\ninput a\ninput b\ncell u INV_X1 A=a ZN=b\n",    # two drivers
    "net a 1\nnet b 1\ninput a\n",                                      # undriven net
    "net a 1\ninput a\nwire a 2\n",                                     # unknown statement
])
def test_malformed_netlists_rejected(bad, library_text):
    with pytest.raises(ValueError):
        Oracle(bad, library_text)
