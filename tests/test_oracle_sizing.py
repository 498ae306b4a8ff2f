"""Pins of the oracle's sizing score (Eq. 8): the hand-worked example (golden/hand_sizing.txt)
and properties that fix each factor independently."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests.golden.fixtures import load


def test_sizing_scores_hand():
    lib, net, v = load("hand_sizing.txt")
    o = Oracle(net, lib)
    K = v["K"][0]
    for mode, key in [(0, "score0_K2"), (1, "score1_K2")]:
        s, psw = o.sizing_scores(np.array(v["sp_in"]), np.array(v["tr_in"]), mode)
        np.testing.assert_allclose(psw, np.array(v["psw_K"]) * K, rtol=1e-13)
        np.testing.assert_allclose(s, np.array(v[key]) * K * K, rtol=1e-12)


def test_scores_of_a_sink_cell_are_local(library_text):
    """A cell whose output feeds nothing: its SP adjoint is its own local term K C (2 - 4 SP),
    so mode 1 gives |K C| P_sw = K C * K TR C and mode 0 |K C (2 - 4 SP)| K TR C."""
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 5, 1)
    sp, tr = sp[:, 0].astype(np.float64), tr[:, 0].astype(np.float64)
    K = 0.32e-6
    spn, trn = o.forward(sp, tr, 0)
    cl = o.cload()
    y = o.cell_outs()
    # nets with no sinks: no cell reads them
    lines = [ln.split() for ln in text.splitlines() if ln.startswith("cell ")]
    read = set()
    for ln in lines:
        for t in ln[3:]:
            pin, n = t.split("=")
            if pin not in ("Z", "ZN"):
                read.add(n)
    names = [ln.split()[1] for ln in text.splitlines() if ln.startswith("net ")]
    sink_free = [i for i, c in enumerate(y) if names[c] not in read]
    assert sink_free
    s0, psw = o.sizing_scores(sp, tr, 0)
    s1, _ = o.sizing_scores(sp, tr, 1)
    for i in sink_free:
        n = y[i]
        assert psw[i] == pytest.approx(K * trn[n] * cl[n], rel=1e-14)
        assert s0[i] == pytest.approx(abs(K * cl[n] * (2 - 4 * spn[n])) * psw[i], rel=1e-10, abs=1e-40)
        assert s1[i] == pytest.approx(K * cl[n] * psw[i], rel=1e-10)


def test_score_scales_with_k_squared(library_text):
    """Both factors are proportional to K = 1/2 Vdd^2 f: the score scales with K^2."""
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 6, 1)
    a, _ = o.sizing_scores(sp[:, 0], tr[:, 0], 0, vdd=0.8)
    b, _ = o.sizing_scores(sp[:, 0], tr[:, 0], 0, vdd=1.6)
    np.testing.assert_allclose(b, 16 * a, rtol=1e-12)
