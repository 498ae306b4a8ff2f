"""Oracle simulation pins (Sec. III-C, Eq. 4; Sec. III-D, Eq. 5).

* Philox4x32-10 equals Triton's independent implementation (tl.philox, run by Triton's CPU
  interpreter) on random counters and keys.
* Startpoint Markov chains: the initial bits are Binomial(64, SP) and, by the Markov property,
  the number of 1->0 (0->1) steps given the number of visits to 1 (0) is binomial with
  p10 = TR / 2SP (p01 = TR / 2(1-SP)); the z-scores over thousands of startpoints must look
  standard normal.
* Every cell's words equal the Boolean function of its fanin words (bitwise, all lanes).
* Toggle and ones counts equal the PopCount definitions on the words.
* Fanout-free circuits with temporally independent inputs (TR = 2SP(1-SP)): every net is
  i.i.d. Bernoulli(P) in time, so the toggle count has mean 64 (T-1) 2P(1-P) and the exact
  variance of a 1-dependent sum; all z-scores stay within 5.5, hence beta ~ 1.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle.oracle import Oracle, philox4x32_10
from paper_2608_03778_gb300 import netgen
from tests import _gates as G
from tests.test_oracle_bruteforce import random_tree

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_triton(tmp_path):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(2024)
    ctr = rng.integers(0, 2 ** 32, (6, 64, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0, :4] = 0
    ctr[1, :4] = 0xFFFFFFFF
    keys = rng.integers(0, 2 ** 32, (6, 2), dtype=np.uint64).astype(np.uint32)
    keys[0] = 0
    inp, outp = tmp_path / "in.npz", tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, keys=keys)
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_philox_triton.py"), str(inp), str(outp)],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip(f"triton interpreter unavailable: {r.stderr[-300:]}")
    got = np.load(outp)
    want = np.stack([np.stack([philox4x32_10(ctr[b, i], keys[b]) for i in range(64)]) for b in range(6)])
    np.testing.assert_array_equal(got, want)


@pytest.fixture(scope="module")
def mid_sim(library_text):
    spec = netgen.WORKLOADS["mid"]
    text = netgen.netlist_text(spec)
    o = Oracle(text, library_text)
    sp_in, tr_in = netgen.scenario_inputs(o.n_start, 2000)
    tg, on, words = o.simulate(sp_in[:, 0], tr_in[:, 0], 42, 64, want_words=True)
    return text, o, sp_in[:, 0], tr_in[:, 0], tg, on, words


def lane_bits(words):
    """[nets, T] uint64 -> [nets, 64 lanes, T] 0/1"""
    b = (words[:, None, :] >> np.arange(64, dtype=np.uint64)[None, :, None]) & np.uint64(1)
    return b.astype(np.int8)


def zscores(k, n, p):
    ok = (n > 0) & (p > 0) & (p < 1)
    return (k[ok] - n[ok] * p[ok]) / np.sqrt(n[ok] * p[ok] * (1 - p[ok]))


def test_markov_startpoints(mid_sim):
    text, o, sp_in, tr_in, tg, on, words = mid_sim
    sn = o.start_nets()
    bits = lane_bits(words[sn])                              # [ns, 64, T]
    sp, tr = sp_in.astype(np.float64), tr_in.astype(np.float64)
    p10 = np.clip(np.where(sp > 0, tr / (2 * sp), 0), 0, 1)
    p01 = np.clip(np.where(sp < 1, tr / (2 * (1 - sp)), 0), 0, 1)
    z0 = zscores(bits[:, :, 0].sum(1).astype(float), np.full(len(sp), 64.0), sp)
    cur, nxt = bits[:, :, :-1], bits[:, :, 1:]
    n1 = (cur == 1).sum((1, 2)).astype(float)
    n0 = (cur == 0).sum((1, 2)).astype(float)
    n10 = ((cur == 1) & (nxt == 0)).sum((1, 2)).astype(float)
    n01 = ((cur == 0) & (nxt == 1)).sum((1, 2)).astype(float)
    for z in [z0, zscores(n10, n1, p10), zscores(n01, n0, p01)]:
        assert len(z) > 8000
        assert np.abs(z).max() < 5.5
        assert abs(z.mean()) < 0.05
        assert 0.95 < z.std() < 1.05


def test_cell_words_are_boolean_functions(mid_sim):
    text, o, sp_in, tr_in, tg, on, words = mid_sim
    sn = o.start_nets()
    want = G.boolean_eval(text, [words[n] for n in sn])
    np.testing.assert_array_equal(np.stack(list(want)), words)


def test_popcount_definitions(mid_sim):
    text, o, sp_in, tr_in, tg, on, words = mid_sim
    bits = lane_bits(words)
    np.testing.assert_array_equal(on, bits.sum((1, 2)))
    np.testing.assert_array_equal(tg, (bits[:, :, 1:] != bits[:, :, :-1]).sum((1, 2)))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_temporally_independent_trees(seed, library_text):
    rng = np.random.default_rng(100 + seed)
    text = random_tree(rng, 18)
    o = Oracle(text, library_text)
    sp_in = rng.uniform(0.1, 0.9, o.n_start).astype(np.float32)
    tr_in = (2 * sp_in.astype(np.float64) * (1 - sp_in.astype(np.float64))).astype(np.float32)
    T = 64
    tg, on = o.simulate(sp_in, tr_in, 7 + seed, T)
    sp, tr = o.forward(sp_in, tr_in)
    cells = o.cell_outs()
    P = sp[cells]
    tau = 2 * P * (1 - P)
    c = P * (1 - P) - tau ** 2
    var = 64 * ((T - 1) * tau * (1 - tau) + 2 * (T - 2) * c)
    ok = var > 0
    z = (tg[cells][ok] - 64 * (T - 1) * tau[ok]) / np.sqrt(var[ok])
    assert np.abs(z).max() < 5.5
    beta, trh = o.hybrid(tr, tg, T)
    assert np.abs(beta[cells][tau > 0.2] - 1).max() < 0.1


def test_hybrid_special_cases(library_text):
    # constant startpoints: SP 0 or 1 means TR_model = 0 and no toggles -> beta = 1 (reading R5)
    text = "net a 1\nnet b 1\nnet y 1\ninput a\ninput b\ncell u AND2_X1 A1=a A2=b ZN=y\n"
    o = Oracle(text, library_text)
    sp_in = np.array([0.0, 1.0], np.float32)
    tr_in = np.array([0.0, 0.0], np.float32)
    tg, on = o.simulate(sp_in, tr_in, 1, 64)
    assert (tg == 0).all() and on[0] == 0 and on[1] == 64 * 64
    sp, tr = o.forward(sp_in, tr_in)
    beta, trh = o.hybrid(tr, tg)
    np.testing.assert_array_equal(beta, 1.0)
    # a net whose model TR is 0 but which toggles gets beta_max; its hybrid TR stays 0
    beta, trh = o.hybrid(np.array([0.0, 0.5, 0.25]), np.array([10, 0, 4032], np.uint32), 64, 0.1, 10.0)
    assert beta[0] == 10.0 and trh[0] == 0.0
    assert beta[1] == 0.1                       # clipped below
    assert beta[2] == 4.0 and trh[2] == 1.0     # TR_acc / TR_model = 1 / 0.25


def test_flip_probabilities_below_the_draw_resolution(library_text):
    """Reading R7 draws 16-bit numbers against floor(p 2^16): a flip probability in (0, 2^-16)
    rounds to threshold 0 and never fires, so a chain whose p10 and p01 both lie there keeps its
    initial bits (toggles 0) and its beta is beta_min (TR_model > 0, TR_acc = 0); a probability of
    exactly 2^-16 keeps threshold 1, i.e. fires with probability 2^-16 per draw (binomial count
    over 4,096 chains)."""
    n = 4096
    lines = [f"net i{k} 1" for k in range(n)] + ["net y 1"] + [f"input i{k}" for k in range(n)]
    lines.append("cell u BUF_X1 A=i0 Z=y")
    o = Oracle("\n".join(lines) + "\n", library_text)
    sn = o.start_nets()
    below = np.nextafter(np.float32(2.0 ** -16), np.float32(0))
    sp = np.full(n, 0.5, np.float32)
    tr = np.full(n, below, np.float32)          # p10 = p01 = tr / (2 * 0.5) = tr < 2^-16
    tg, on, words = o.simulate(sp, tr, 5, 64, want_words=True)
    assert (tg[sn] == 0).all()
    assert (words[sn] == words[sn][:, :1]).all()     # every lane keeps its initial bit
    z = zscores(on[sn].astype(float) / 64, np.full(n, 64.0), np.full(n, 0.5))
    assert np.abs(z).max() < 5.5                 # initial states still Bernoulli(SP)
    _, trm = o.forward(sp, tr)
    beta, trh = o.hybrid(trm, tg, 64, 0.1, 10.0)
    np.testing.assert_array_equal(beta[sn], 0.1)
    # exactly 2^-16: 4,096 chains x 64 lanes x 63 steps draws, each a flip with probability 2^-16
    tr[:] = np.float32(2.0 ** -16)
    tg, on = o.simulate(sp, tr, 5, 64)
    draws = n * 64 * 63
    z = (tg[sn].sum() - draws * 2.0 ** -16) / np.sqrt(draws * 2.0 ** -16)
    assert tg[sn].sum() > 0 and abs(z) < 5.5
    # SP below 2^-16: the initial state is always 0 as well
    sp[:] = np.float32(1e-5)
    tr[:] = np.float32(1e-5)                     # p01 = 5e-6
    tg, on = o.simulate(sp, tr, 5, 64)
    assert (tg[sn] == 0).all() and (on[sn] == 0).all()
