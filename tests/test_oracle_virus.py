"""Pins of the oracle's batched scenarios, ascent (Algorithm 4) and P_virus (Eq. 3).

Each check fixes the oracle by something other than itself: a hand-worked
example (golden/hand_virus.txt), an independent Boolean evaluator
(tests/_gates.py), closed forms on circuits whose answer is known, and the
ascent property of a small step.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests import _gates as G
from tests.golden.fixtures import load

K = 0.5 * 0.8 * 0.8 * 1e9 * 1e-15


@pytest.fixture(scope="module")
def hand():
    lib, net, v = load("hand_virus.txt")
    return Oracle(net, lib), v


@pytest.fixture(scope="module")
def small():
    spec = netgen.WORKLOADS["small"]
    text = netgen.netlist_text(spec)
    return text, Oracle(text, netgen.library_text())


def test_virus_hand(hand):
    o, v = hand
    sp = np.array([v["virus_sp_a"], v["virus_sp_b"]], np.float32)
    pv, v0 = o.p_virus(sp)
    np.testing.assert_array_equal(v0, np.array([v["virus_v0_a"], v["virus_v0_b"]], np.uint8))
    np.testing.assert_allclose(pv, v["p_virus"], rtol=1e-15)


def test_proxy_and_gradient_hand(hand):
    o, v = hand
    sp = np.array(v["sp_in"])
    assert o.proxy(sp, np.zeros(2), tr_mode=1) == pytest.approx(v["proxy"][0], rel=1e-15)
    g = o.backward(sp, np.zeros(2), None, 0, 1)["grad_sp_in"] / K
    np.testing.assert_allclose(g, v["proxy_grad"], rtol=1e-13)


@pytest.mark.parametrize("eta,key", [(0.1, "step_eta_0.1"), (1.0, "step_eta_1")])
def test_ascent_step_hand(hand, eta, key):
    o, v = hand
    sp, _ = o.ascent(np.array(v["sp_in"])[:, None], np.zeros((2, 1)), 1, eta, tr_mode=1)
    np.testing.assert_allclose(sp[:, 0], v[key], rtol=1e-13)


def test_logic_words_are_boolean_functions(small):
    text, o = small
    rng = np.random.default_rng(5)
    words = rng.integers(0, 2**63, o.n_start, dtype=np.uint64) ^ rng.integers(0, 2, o.n_start, dtype=np.uint64) << 63
    want = G.boolean_eval(text, list(words))
    np.testing.assert_array_equal(o.logic(words), np.stack(list(want)).astype(np.uint64))


def test_p_virus_definition(small):
    """Eq. 3 term by term: independent Boolean evaluation of v0 and v1 = not v0."""
    text, o = small
    sp, _ = netgen.scenario_inputs(o.n_start, 77, 5)
    sp[:3, 0] = 0.5          # ties decide v0 = 1
    sp[3:6, 0] = np.nextafter(np.float32(0.5), np.float32(0))
    pv, v0 = o.p_virus(sp)
    cl = o.cload()
    for s in range(sp.shape[1]):
        b0 = (sp[:, s] >= np.float32(0.5)).astype(np.int64)
        assert list(v0[:, s]) == list(b0)
        a = G.boolean_eval(text, list(b0))
        b = G.boolean_eval(text, list(1 - b0))
        want = math.fsum(cl[n] for n in range(len(cl)) if int(a[n]) != int(b[n]))
        assert pv[s] == want


def test_p_virus_inverter_chain():
    """Every net of an inverter/buffer chain toggles when its input does: P_virus = sum C_load."""
    lib = netgen.library_text()
    lines = ["net x0 1.0", "input x0"]
    for i in range(6):
        g = "INV" if i % 2 == 0 else "BUF"
        pin = "A"
        out = G.BOOL[g][1]
        lines += [f"net x{i + 1} {0.5 + 0.25 * i}", f"cell u{i} {g}_X2 {pin}=x{i} {out}=x{i + 1}"]
    lines.append("output x6")
    o = Oracle("\n".join(lines) + "\n", lib)
    for p in (0.2, 0.9):
        pv, _ = o.p_virus(np.array([[p]], np.float32))
        assert pv[0] == pytest.approx(float(np.sum(o.cload())), rel=1e-15)


def test_p_virus_xor_of_toggling_inputs(library_text):
    """XOR of two inputs that both flip does not flip: only the inputs count."""
    net = ("net a 1.0\nnet b 2.0\nnet y 0.5\ninput a\ninput b\n"
           "cell u1 XOR2_X1 A=a B=b Z=y\noutput y\n")
    o = Oracle(net, library_text)
    pv, _ = o.p_virus(np.array([[0.7], [0.2]], np.float32))
    cl = o.cload()
    assert pv[0] == pytest.approx(cl[0] + cl[1], rel=1e-15)


def test_ascent_isolated_net_closed_form(library_text):
    """a -> BUF -> y: proxy = (C_a + C_y) 2P(1-P), so P <- clip(P + eta (C_a + C_y)(2 - 4P))."""
    net = "net a 1.5\nnet y 0.7\ninput a\ncell u1 BUF_X1 A=a Z=y\noutput y\n"
    o = Oracle(net, library_text)
    c = float(np.sum(o.cload()))
    for p0, eta in [(0.1, 0.05), (0.93, 0.02), (0.3, 0.6)]:
        p = p0
        for _ in range(7):
            p = min(max(p + eta * c * (2 - 4 * p), 0.0), 1.0)
        sp, _ = o.ascent(np.array([[p0]]), np.zeros((1, 1)), 7, eta, tr_mode=1)
        assert sp[0, 0] == pytest.approx(p, rel=1e-12, abs=1e-15)


def test_ascent_tr_mode0_moves_tr_by_load(small):
    """In tr_mode 0 dProxy/dTR_k = C_load,k, so one step adds eta C_load (then clips)."""
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 5, 2)
    _, tr1 = o.ascent(sp.astype(np.float64), tr.astype(np.float64), 1, 0.0, 0.03, tr_mode=0)
    cl = o.cload()[o.start_nets()]
    np.testing.assert_allclose(tr1, np.clip(tr + 0.03 * cl[:, None], 0, 1), rtol=1e-12)


def test_ascent_small_steps_increase_the_proxy(small):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 9, 1)
    x = sp.astype(np.float64)
    prev = o.proxy(x[:, 0], tr[:, 0], 1)
    for _ in range(5):
        x, _ = o.ascent(x, tr.astype(np.float64), 1, 1e-3, tr_mode=1)
        assert np.all((x >= 0) & (x <= 1))
        cur = o.proxy(x[:, 0], tr[:, 0], 1)
        assert cur >= prev
        prev = cur


def test_backward_batch_is_weighted_per_scenario(small):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 3, 3)
    w = np.array([1.0, -2.5, 0.25])
    gb = o.backward_batch(sp, tr, w, 0)
    for s in range(3):
        g = o.backward(sp[:, s], tr[:, s], None, 0, 0)
        np.testing.assert_array_equal(gb["grad_sp_in"][:, s], w[s] * g["grad_sp_in"])
    np.testing.assert_allclose(gb["grad_pincap_sum"], gb["grad_pincap"].sum(axis=1), rtol=1e-15)
