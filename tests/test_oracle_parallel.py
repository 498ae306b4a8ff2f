"""The oracle's level-parallel variants (the all-core CPU baseline) against the serial oracle:
forward SP/TR and the simulation words bitwise equal (the same per-cell arithmetic, cells of one
level in parallel), the adjoint within rounding (each net gathers over its sink pins instead of
the serial scatter), in every gradient and TR mode, on a reconvergent netlist and on a library
with repeated nets, constants and 4-input cells."""
import numpy as np
import pytest

from oracle.oracle import Oracle, threads
from paper_2608_03778_gb300 import netgen
from tests._netlists import custom_case


def close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(b), 1e-3 * np.abs(b).max(initial=0)) + 1e-300)


def check(o, sp, tr):
    for tr_mode in (0, 1):
        a = o.forward(sp, tr, tr_mode, want_sq=True)
        b = o.forward(sp, tr, tr_mode, want_sq=True, parallel=True)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    tg, on, w = o.simulate(sp, tr, 9, 33, want_words=True)
    tg2, on2, w2 = o.simulate(sp, tr, 9, 33, want_words=True, parallel=True)
    np.testing.assert_array_equal(w, w2)
    np.testing.assert_array_equal(tg, tg2)
    np.testing.assert_array_equal(on, on2)
    _, trm = o.forward(sp, tr)
    beta, _ = o.hybrid(trm, tg, 33)
    for grad_mode in (0, 1, 2):
        for tr_mode in (0, 1):
            b = beta if grad_mode else None
            g1 = o.backward(sp, tr, b, grad_mode, tr_mode)
            g2 = o.backward(sp, tr, b, grad_mode, tr_mode, parallel=True)
            for k in g1:
                assert close(g2[k], g1[k]), (k, grad_mode, tr_mode)


def test_parallel_matches_serial_generated(library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    check(o, sp[:, 0].astype(np.float64), tr[:, 0].astype(np.float64))


@pytest.mark.parametrize("seed", [1, 2])
def test_parallel_matches_serial_custom(seed):
    rng = np.random.default_rng(seed)
    text, lib = custom_case(rng, n_cells=200)
    o = Oracle(text, lib)
    sp = rng.uniform(0, 1, o.n_start).astype(np.float32).astype(np.float64)
    tr = (rng.uniform(0, 1, o.n_start) * 2 * np.minimum(sp, 1 - sp)).astype(np.float32).astype(np.float64)
    check(o, sp, tr)


def test_thread_count():
    assert threads() >= 1
