"""Pins of the oracle's lag-one mode (every net carries SP and the probability T that two
consecutive values differ; a cell's T is its exact toggle probability under spatial
independence).

* single gates: closed forms worked out by hand;
* fanout-free trees: exact toggle probability of every net by enumerating all joint
  input histories (x_t, x_{t+1}) with an independent Boolean evaluator;
* temporally independent inputs (T = 2P(1-P)) on a reconvergent netlist: Eq. 2 on every net;
* the bit-parallel Markov simulator on trees: toggle counts within statistical bounds;
* gradients: central finite differences; cap gradients: exact linearity in the caps.
"""
import itertools

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests import _gates as G
from tests.test_oracle_bruteforce import random_tree

K = 0.5 * 0.8 * 0.8 * 1e9 * 1e-15


def feasible(rng, n):
    p = rng.uniform(0.05, 0.95, n)
    t = rng.uniform(0, 1, n) * 2 * np.minimum(p, 1 - p)
    return p, t


def one_cell(gate):
    ins, out, _ = G.BOOL[gate]
    lines = []
    for i, pin in enumerate(ins):
        lines += [f"net i{i} 1.0", f"input i{i}"]
    lines += ["net y 1.0", f"cell u0 {gate}_X1 " + " ".join(f"{p}=i{i}" for i, p in enumerate(ins)) + f" {out}=y",
              "output y"]
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("seed", range(5))
def test_single_gate_closed_forms(library_text, seed):
    rng = np.random.default_rng(seed)
    (pa, pb), (ta, tb) = feasible(rng, 2)
    q11 = lambda p, t: p - t / 2  # noqa: E731
    want = {
        "INV": ta, "BUF": ta,
        "XOR2": ta * (1 - tb) + tb * (1 - ta), "XNOR2": ta * (1 - tb) + tb * (1 - ta),
        # AND: the output is 1 at t with prob pa pb, and stays 1 with prob q11(a) q11(b)
        "AND2": 2 * (pa * pb - q11(pa, ta) * q11(pb, tb)), "NAND2": 2 * (pa * pb - q11(pa, ta) * q11(pb, tb)),
        "OR2": 2 * ((1 - pa) * (1 - pb) - q11(1 - pa, ta) * q11(1 - pb, tb)),
        "NOR2": 2 * ((1 - pa) * (1 - pb) - q11(1 - pa, ta) * q11(1 - pb, tb)),
    }
    for gate, t_want in want.items():
        o = Oracle(one_cell(gate), library_text)
        k = len(G.BOOL[gate][0])
        _, tr = o.forward_lag1(np.array([pa, pb][:k]), np.array([ta, tb][:k]))
        assert tr[-1] == pytest.approx(t_want, rel=1e-12, abs=1e-15), gate


@pytest.mark.parametrize("seed", range(6))
def test_fanout_free_trees_are_exact(library_text, seed):
    """Every net of a fanout-free circuit: T equals the enumerated toggle probability."""
    rng = np.random.default_rng(100 + seed)
    text = random_tree(rng, int(rng.integers(3, 8)))
    o = Oracle(text, library_text)
    n = o.n_start
    p, t = feasible(rng, n)
    _, tr = o.forward_lag1(p, t)
    # all joint input states (x_t, x_{t+1}), each startpoint independently
    states = np.array(list(itertools.product(range(4), repeat=n)), np.int64)   # [4^n, n], digit 2a+b
    w = np.stack([np.array([1 - p[i] - t[i] / 2, t[i] / 2, t[i] / 2, p[i] - t[i] / 2])[states[:, i]]
                  for i in range(n)], axis=1).prod(axis=1)
    a = [(states[:, i] >> 1) for i in range(n)]
    b = [(states[:, i] & 1) for i in range(n)]
    va = G.boolean_eval(text, a)
    vb = G.boolean_eval(text, b)
    want = np.array([np.sum(w * (np.asarray(x) != np.asarray(y))) for x, y in zip(va, vb)])
    np.testing.assert_allclose(tr, want, rtol=1e-12, atol=1e-15)


def test_temporally_independent_inputs_give_eq2(library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, _ = netgen.scenario_inputs(o.n_start, 3, 1)
    p = sp[:, 0].astype(np.float64)
    s1, t1 = o.forward_lag1(p, 2 * p * (1 - p))
    s2, t2, q2 = o.forward(p, 2 * p * (1 - p), 1, want_sq=True)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_allclose(t1, t2, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("seed", range(3))
def test_markov_simulation_agrees_on_trees(library_text, seed):
    """The simulator's chains are stationary with the lag-one law; on a tree every net's toggle
    fraction over 64 x 63 transitions estimates T."""
    rng = np.random.default_rng(200 + seed)
    text = random_tree(rng, 7)
    o = Oracle(text, library_text)
    p, t = feasible(rng, o.n_start)
    p32, t32 = p.astype(np.float32), t.astype(np.float32)
    _, tr = o.forward_lag1(p32.astype(np.float64), t32.astype(np.float64))
    T = 64
    z = []
    for sim_seed in range(8):
        tg, _ = o.simulate(p32, t32, seed=1000 * seed + sim_seed, T=T)
        frac = tg / (64.0 * (T - 1))
        # 64 independent chains; within a chain successive transitions are correlated, so the
        # variance bound is inflated 8-fold over the binomial one
        sd = np.sqrt(8 * np.maximum(tr * (1 - tr), 1e-6) / (64.0 * (T - 1)))
        z.append((frac - tr) / sd)
    z = np.array(z)
    assert np.abs(z).max() < 5


def test_lag1_gradients_central_fd(library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    rng = np.random.default_rng(9)
    p, t = feasible(rng, o.n_start)
    g = o.backward_lag1(p, t)
    cl = o.cload()

    def power(pp, tt):
        return K * float(np.sum(o.forward_lag1(pp, tt)[1] * cl))

    h = 1e-6
    idx = rng.choice(o.n_start, 12, replace=False)
    for k in idx:
        for key, arr in [("grad_sp_in", p), ("grad_tr_in", t)]:
            up, dn = arr.copy(), arr.copy()
            up[k] += h
            dn[k] -= h
            fd = (power(up, t) - power(dn, t)) / (2 * h) if key == "grad_sp_in" else \
                (power(p, up) - power(p, dn)) / (2 * h)
            scale = np.abs(g[key]).max()
            assert abs(g[key][k] - fd) <= 1e-6 * abs(fd) + 1e-7 * scale, (key, k)


def test_lag1_cap_gradients_are_exact_linear(library_text):
    """The power is linear in each cell's pin cap with slope K * sum of its inputs' T."""
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    rng = np.random.default_rng(4)
    p, t = feasible(rng, o.n_start)
    g = o.backward_lag1(p, t)
    base = K * float(np.sum(o.forward_lag1(p, t)[1] * o.cload()))
    refs = [ln.split()[2] for ln in text.splitlines() if ln.startswith("cell ")]
    caps = {"X1": 0.8, "X2": 1.6, "X4": 3.2}
    for c in rng.choice(o.n_cells, 5, replace=False):
        o2 = Oracle(text, library_text)
        o2.set_pincap(int(c), 10.0)
        new = K * float(np.sum(o2.forward_lag1(p, t)[1] * o2.cload()))
        dc = 10.0 - caps[refs[c].rsplit("_", 1)[1]]
        assert new - base == pytest.approx(g["grad_pincap"][c] * dc, rel=1e-9, abs=1e-20)
