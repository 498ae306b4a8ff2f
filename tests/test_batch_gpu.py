"""Batched scenarios, the autograd Function and the power-virus search on the GPU,
against the FP64 oracle (each scenario an independent oracle run).

Tolerances as for one scenario: SP/TR 1e-5 absolute, power 1e-6 relative,
gradients |g - g*| <= 1e-4 max(|g*|, 1e-3 max|g*|); the thresholded vectors
bit-exact, and P_virus (an FP64 sum of the nets' binary32 C_load, the same
caps the power uses, against the oracle's binary64 caps) 1e-7 relative, while
a single net counted wrongly would move it by more than 1e-4.
"""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 0.5 * 0.8 * 0.8 * 1e9 * 1e-15


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp as _dp
    return _dp


@pytest.fixture(scope="module")
def ctx(dp):
    c = dp.dp_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    dp.dp_destroy(c)


@pytest.fixture(scope="module")
def small():
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    return text, Oracle(text, netgen.library_text())


def grad_close(g, g_star, axis=None):
    g, g_star = np.asarray(g, np.float64), np.asarray(g_star, np.float64)
    if g_star.size == 0:
        return True
    floor = 1e-3 * np.abs(g_star).max(axis=axis, keepdims=axis is not None)
    bad = np.abs(g - g_star) > 1e-4 * np.maximum(np.abs(g_star), floor)
    if bad.any():
        r = np.abs(g - g_star) / np.maximum(np.abs(g_star), floor + 1e-300)
        i = np.unravel_index(np.argmax(r), r.shape)
        print(f"worst at {i}: {g[i]} vs {g_star[i]}")
    return not bad.any()


def run_batch(dp, ctx, d, sp, tr, cfg, weights=None, reduce=0):
    """dp_set_inputs_batch, dp_propagate, powers, weighted backward, nets; host buffers."""
    info = dp.dp_design_info(d)
    ns, nc, nn = info.n_start, info.n_cells, info.n_nets
    S = sp.shape[1]
    dp.dp_set_inputs_batch(ctx, d, np.ascontiguousarray(sp), np.ascontiguousarray(tr), S)
    dp.dp_propagate(ctx, d, cfg)
    out = {"power": np.zeros(S)}
    dp.dp_get_power(ctx, d, out["power"])
    rows = {"grad_sp_in": ns, "grad_tr_in": ns, "grad_pincap": nc, "grad_cload": nn}
    for k, n in rows.items():
        out[k] = np.zeros((n,) if reduce and k in ("grad_pincap", "grad_cload") else (n, S), np.float32)
    dp.dp_backward_weighted(ctx, d, cfg, None if weights is None else np.ascontiguousarray(weights, np.float64),
                            reduce, out["grad_sp_in"], out["grad_tr_in"], out["grad_pincap"], out["grad_cload"])
    out["sp"] = np.zeros((nn, S), np.float32)
    out["tr"] = np.zeros((nn, S), np.float32)
    dp.dp_get_nets(ctx, d, out["sp"], out["tr"])
    return out


def check_scenarios(o, g, sp, tr, cfg, scen, weights=None):
    w = np.ones(sp.shape[1]) if weights is None else weights
    for s in scen:
        spf, trf = o.forward(sp[:, s], tr[:, s], cfg.tr_mode)
        assert np.abs(g["sp"][:, s] - spf).max(initial=0) <= 1e-5, s
        assert np.abs(g["tr"][:, s] - trf).max(initial=0) <= 1e-5, s
        assert g["power"][s] == pytest.approx(o.power(trf, cfg.vdd, cfg.fclk), rel=1e-6, abs=1e-30), s
        ref = o.backward(sp[:, s], tr[:, s], None, 0, cfg.tr_mode, cfg.vdd, cfg.fclk)
        for k in ["grad_sp_in", "grad_tr_in", "grad_pincap", "grad_cload"]:
            if g[k].ndim == 2:
                assert grad_close(g[k][:, s], w[s] * ref[k]), (k, s)


@pytest.mark.parametrize("tr_mode", [0, 1])
@pytest.mark.parametrize("S", [1, 37, 130])
def test_small_batch_parity(dp, ctx, small, tr_mode, S):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 1000, S)
    cfg = dp.config(grad_mode=0, tr_mode=tr_mode)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
    finally:
        dp.dp_design_free(d)
    check_scenarios(o, g, sp, tr, cfg, range(S))


def test_weights_and_scenario_sums(dp, ctx, small):
    text, o = small
    S = 45
    sp, tr = netgen.scenario_inputs(o.n_start, 2000, S)
    w = np.random.default_rng(1).uniform(-2, 3, S)
    cfg = dp.config(grad_mode=0, tr_mode=0)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg, weights=w)
        gr = run_batch(dp, ctx, d, sp, tr, cfg, weights=w, reduce=1)
    finally:
        dp.dp_design_free(d)
    check_scenarios(o, g, sp, tr, cfg, range(S), weights=w)
    ref = o.backward_batch(sp, tr, w, 0)
    assert grad_close(gr["grad_pincap"], ref["grad_pincap_sum"])
    assert grad_close(gr["grad_cload"], ref["grad_cload_sum"])
    # the FP64 scenario sum of the binary32 per-scenario outputs, up to the final rounding
    np.testing.assert_allclose(gr["grad_pincap"], g["grad_pincap"].astype(np.float64).sum(axis=1),
                               rtol=2e-6, atol=1e-6 * np.abs(g["grad_pincap"]).max())


@pytest.mark.parametrize("S", [70, 72])
def test_shapes_give_identical_bits(dp, ctx, small, S):
    """Every launch shape gives the same bits: scenario widths, cells per block, and 1, 2 or 4
    scenarios per thread (a v that does not divide S falls back to 1)."""
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 3000, S)
    cfg = dp.config(grad_mode=0, tr_mode=0)
    results = []
    # (bx, by) or (bx, by, v) for both passes, or one shape per pass; v scenarios per thread
    for shape in ["32,4", "64,2,32,8", "128,1", "256,1,64,4", "64,2,2", "128,1,2,32,8,1", "32,8,1,128,2,2",
                  "32,4,4", "64,2,4,128,1,2", "128,1,4"]:
        os.environ["DP_BATCH_SHAPE"] = shape
        try:
            d = dp.dp_design_load(ctx, text, netgen.library_text())
            try:
                g = run_batch(dp, ctx, d, sp, tr, cfg)
                a = [int(x) for x in shape.split(",")]
                want = {2: a + [1] + a + [1], 3: a + a, 4: a[:2] + [1] + a[2:] + [1], 6: a}[len(a)]
                fwd, bwd, _ = dp.dp_batch_tuning(d)
                assert list(fwd) + list(bwd) == want
            finally:
                dp.dp_design_free(d)
        finally:
            del os.environ["DP_BATCH_SHAPE"]
        results.append(g)
    for g in results[1:]:
        for k in g:
            np.testing.assert_array_equal(g[k], results[0][k], err_msg=k)


@pytest.mark.parametrize("tr_mode", [0, 1, 2])
def test_narrow_batches_match_wide_ones(dp, ctx, small, tr_mode):
    """A batch narrower than the tuned scenario width runs with the width cut to the power of
    two covering it (more cells per block); each scenario gives the same bits as the same
    scenario inside a wide batch."""
    text, o = small
    S = 70
    sp, tr = netgen.scenario_inputs(o.n_start, 3100, S)
    cfg = dp.config(grad_mode=0, tr_mode=tr_mode)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        wide = run_batch(dp, ctx, d, sp, tr, cfg)
        for cols in ([0], [69], [3, 4, 5], list(range(10, 27))):
            g = run_batch(dp, ctx, d, np.ascontiguousarray(sp[:, cols]), np.ascontiguousarray(tr[:, cols]), cfg)
            for k in g:
                want = wide[k][:, cols] if wide[k].ndim == 2 else wide[k][cols]
                np.testing.assert_array_equal(g[k], want, err_msg=f"{k} {cols}")
    finally:
        dp.dp_design_free(d)


def test_autotuner_picks_a_candidate(dp, ctx, small):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 4000, 96)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        dp.dp_set_inputs_batch(ctx, d, sp, tr, 96)
        fwd, bwd, ms = dp.dp_batch_tuning(d)
    finally:
        dp.dp_design_free(d)
    for bx, by, v in (fwd, bwd):
        assert bx in (32, 64, 128, 256, 512) and by >= 1 and bx * by <= 1024 and v in (1, 2, 4)
    assert ms[0] > 0 and ms[1] > 0


def test_single_and_batched_paths_agree(dp, ctx, small):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 5000, 1)
    cfg = dp.config(grad_mode=0, tr_mode=0)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        gb = run_batch(dp, ctx, d, sp, tr, cfg)
        dp.dp_set_inputs(ctx, d, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]), 1)
        dp.dp_propagate(ctx, d, cfg)
        p1 = dp.dp_total_power(ctx, d, 0)
        gs = np.zeros(o.n_start, np.float32)
        dp.dp_backward(ctx, d, cfg, gs, None, None, None)
    finally:
        dp.dp_design_free(d)
    assert gb["power"][0] == pytest.approx(p1, rel=1e-6)
    assert grad_close(gb["grad_sp_in"][:, 0], gs)


def test_batch_errors(dp, ctx, small):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 6000, 4)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_inputs_batch(ctx, d, sp, tr, 0)
        assert e.value.name == "DP_EINVAL"
        bad = sp.copy()
        bad[3, 2] = 1.5
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_inputs_batch(ctx, d, bad, tr, 4)
        assert e.value.name == "DP_EINVAL"
        dp.dp_set_inputs(ctx, d, sp, tr, 4)          # n_scen > 1 selects the batched path
        cfg = dp.config(grad_mode=0)
        g = np.zeros((o.n_start, 4), np.float32)
        with pytest.raises(dp.DPError) as e:
            dp.dp_backward(ctx, d, cfg, g)
        assert e.value.name == "DP_ESTATE"
        dp.dp_propagate(ctx, d, cfg)
        for call in [lambda: dp.dp_simulate(ctx, d, cfg), lambda: dp.dp_total_power(ctx, d, 1),
                     lambda: dp.dp_backward(ctx, d, dp.config(grad_mode=1), g),
                     lambda: dp.dp_step(ctx, d, cfg),
                     lambda: dp.dp_get_nets(ctx, d, None, None, np.zeros((o.n_start, 4), np.float32))]:
            with pytest.raises(dp.DPError) as e:
                call()
            assert e.value.name == "DP_EUNSUPPORTED"
        with pytest.raises(dp.DPError) as e:
            dp.dp_backward(ctx, d, dp.config(grad_mode=0, tr_mode=1), g)
        assert e.value.name == "DP_ESTATE"
        dp.dp_set_inputs(ctx, d, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]), 1)
        with pytest.raises(dp.DPError) as e:
            dp.dp_backward_weighted(ctx, d, cfg, np.ones(1), 0, np.zeros(o.n_start, np.float32))
        assert e.value.name == "DP_EUNSUPPORTED"
    finally:
        dp.dp_design_free(d)


def test_mid_512_scenarios_sampled(dp, ctx, library_text):
    """The 120,000-cell netlist x 512 scenarios in one launch, sampled scenarios vs the oracle."""
    text = netgen.netlist_text(netgen.WORKLOADS["mid"])
    o = Oracle(text, library_text)
    S = 512
    sp, tr = netgen.scenario_inputs(o.n_start, 1000, S)
    cfg = dp.config(grad_mode=0, tr_mode=0)
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
        gr = run_batch(dp, ctx, d, sp, tr, cfg, reduce=1)
    finally:
        dp.dp_design_free(d)
    check_scenarios(o, g, sp, tr, cfg, [0, 255, 511])
    for k in ["power", "grad_sp_in", "sp"]:
        np.testing.assert_array_equal(g[k], gr[k])    # the same pass, bit for bit
    sums = g["grad_cload"].astype(np.float64).sum(axis=1)
    np.testing.assert_allclose(gr["grad_cload"], sums, rtol=2e-6, atol=1e-6 * np.abs(sums).max())


def test_virus_eval_parity(dp, ctx, small):
    text, o = small
    S = 70
    sp, _ = netgen.scenario_inputs(o.n_start, 7000, S)
    sp[:5, 3] = 0.5
    sp[5:9, 3] = np.nextafter(np.float32(0.5), np.float32(0))
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        pv = np.zeros(S)
        v0 = np.zeros((o.n_start, S), np.uint8)
        dp.dp_virus_eval(ctx, d, np.ascontiguousarray(sp), S, pv, v0)
    finally:
        dp.dp_design_free(d)
    ref, v0_ref = o.p_virus(sp)
    np.testing.assert_array_equal(v0, v0_ref)
    np.testing.assert_allclose(pv, ref, rtol=1e-7)
    assert 1e-4 * ref.max() < 0.5     # the smallest C_load (a bare wire) is above 0.5 fF


def test_ascent_step_kernel_bits(dp, ctx):
    rng = np.random.default_rng(3)
    n = 100_003
    x = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    g = rng.normal(0, 10, n).astype(np.float32)
    eta = np.float32(0.0137)
    xt = torch.from_numpy(x).cuda()
    gt = torch.from_numpy(g).cuda()
    dp.dp_set_stream(ctx, torch.cuda.current_stream().cuda_stream)
    dp.dp_ascent_step(ctx, xt, gt, n, float(eta))
    torch.cuda.synchronize()
    want = np.clip((x + (eta * g).astype(np.float32)).astype(np.float32), np.float32(0), np.float32(1))
    np.testing.assert_array_equal(xt.cpu().numpy(), want)


def test_autograd_function_matches_oracle(dp, small):
    from paper_2608_03778_gb300 import torch_api as ta
    text, _ = small
    o = Oracle(text, netgen.library_text())     # its pin caps change below
    S = 19
    sp, tr = netgen.scenario_inputs(o.n_start, 8000, S)
    des = ta.Design(text, netgen.library_text())
    try:
        x = torch.from_numpy(sp).cuda().requires_grad_(True)
        t = torch.from_numpy(tr).cuda().requires_grad_(True)
        pin = torch.ones(o.n_cells, dtype=torch.float32, device="cuda")
        pin.copy_(torch.from_numpy(np.array([0.8, 1.6, 3.2], np.float32)[np.arange(o.n_cells) % 3]))
        for c in range(o.n_cells):
            o.set_pincap(c, float(pin[c]))
        pin.requires_grad_(True)
        p = ta.power(des, x, t, pin)
        w = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 2, S)).cuda()
        p.backward(w)
        torch.cuda.synchronize()
        pw = p.detach().cpu().numpy()
        wn = w.cpu().numpy()
        ref = o.backward_batch(sp, tr, wn, 0)
        for s in range(S):
            _, trf = o.forward(sp[:, s], tr[:, s], 0)
            assert pw[s] == pytest.approx(o.power(trf), rel=1e-6)
        assert grad_close(x.grad.cpu().numpy(), ref["grad_sp_in"], axis=0)
        assert grad_close(t.grad.cpu().numpy(), ref["grad_tr_in"], axis=0)
        assert grad_close(pin.grad.cpu().numpy(), ref["grad_pincap_sum"])
        # a second forward between forward and backward: the backward restores its own state
        p1 = ta.power(des, x, t, pin)
        _ = ta.power(des, x * 0 + 0.5, t, pin)
        x.grad = None
        p1.backward(w)
        assert grad_close(x.grad.cpu().numpy(), ref["grad_sp_in"], axis=0)
    finally:
        des.close()


@pytest.mark.parametrize("tr_mode", [1, 0])
def test_power_virus_small(dp, small, tr_mode):
    from paper_2608_03778_gb300 import torch_api as ta
    text, o = small
    S, steps, eta = 9, 12, 0.005
    sp, tr = netgen.scenario_inputs(o.n_start, 9000, S)
    des = ta.Design(text, netgen.library_text())
    try:
        x0, t0 = torch.from_numpy(sp).cuda(), torch.from_numpy(tr).cuda()
        eager = ta.power_virus(des, x0, t0, steps, eta, 0.002, tr_mode=tr_mode, graph=False)
        graphed = ta.power_virus(des, x0, t0, steps, eta, 0.002, tr_mode=tr_mode, graph=True)
    finally:
        des.close()
    assert graphed.graph and not eager.graph
    for k in ["sp", "tr", "v0", "p_virus", "proxy_end"]:
        np.testing.assert_array_equal(getattr(graphed, k).cpu().numpy(), getattr(eager, k).cpu().numpy(), k)
    sp_ref, tr_ref = o.ascent(sp.astype(np.float64), tr.astype(np.float64), steps, eta, 0.002, tr_mode=tr_mode)
    got = eager.sp.cpu().numpy()
    assert np.abs(got - sp_ref).max() <= 1e-4
    assert np.abs(eager.tr.cpu().numpy() - tr_ref).max() <= 1e-4
    assert np.all(eager.proxy_end.cpu().numpy() >= eager.proxy_start.cpu().numpy() - 1e-9)
    # P_virus of the oracle's own end point, wherever no SP lies near the threshold
    pv_ref, _ = o.p_virus(sp_ref.astype(np.float32))
    clear = np.all(np.abs(sp_ref - 0.5) > 1e-3, axis=0)
    assert clear.any()
    np.testing.assert_allclose(eager.p_virus.cpu().numpy()[clear], pv_ref[clear], rtol=1e-7)


# ---- lag-one mode (tr_mode 2) ----

def check_lag1(o, g, sp, tr, scen, vdd=0.8, fclk=1e9):
    K = 0.5 * vdd * vdd * fclk * 1e-15
    cl = o.cload()
    for s in scen:
        spf, trf = o.forward_lag1(sp[:, s].astype(np.float64), tr[:, s].astype(np.float64))
        assert np.abs(g["sp"][:, s] - spf).max(initial=0) <= 1e-5, s
        assert np.abs(g["tr"][:, s] - trf).max(initial=0) <= 1e-5, s
        assert g["power"][s] == pytest.approx(K * float(np.sum(trf * cl)), rel=1e-6), s
        ref = o.backward_lag1(sp[:, s].astype(np.float64), tr[:, s].astype(np.float64), vdd, fclk)
        for k in ["grad_sp_in", "grad_tr_in", "grad_pincap", "grad_cload"]:
            assert grad_close(g[k][:, s], ref[k]), (k, s)


@pytest.mark.parametrize("S", [1, 37])
def test_lag1_parity_small(dp, ctx, small, S):
    text, o = small
    sp, tr = netgen.scenario_inputs(o.n_start, 3100, S)
    cfg = dp.config(grad_mode=0, tr_mode=2)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
    finally:
        dp.dp_design_free(d)
    check_lag1(o, g, sp, tr, range(S))


def test_lag1_custom_cells(dp, ctx):
    """0- to 4-input cells (constants and a 4-input majority-like function) in the lag-one mode."""
    lib = ("cell C0 Z 0.8 0\ncell C1 Z 0.8 1\ncell INV ZN 0.8 !A\ncell AOI211 ZN 1.6 !((A1&A2)|B|C)\n"
           "cell F4 Z 1.2 (A&B)|(C^D)|(A&!D)\ncell MUX2 Z 0.9 (A&!S)|(B&S)\n")
    rng = np.random.default_rng(8)
    lines, nid = [], 0
    for i in range(6):
        lines += [f"net n{nid} 1.0", f"input n{nid}"]
        nid += 1
    cells = [("C0", ["Z"], []), ("C1", ["Z"], []), ("INV", ["ZN"], ["A"]), ("AOI211", ["ZN"], ["A1", "A2", "B", "C"]),
             ("F4", ["Z"], ["A", "B", "C", "D"]), ("MUX2", ["Z"], ["A", "B", "S"])]
    for rep in range(3):
        for ref, (out,), ins in cells:
            pick = rng.choice(nid, len(ins), replace=False)
            lines.append(f"net n{nid} {rng.uniform(0.5, 2):.3f}")
            lines.append(f"cell u{nid} {ref} " + " ".join(f"{p}=n{x}" for p, x in zip(ins, pick)) + f" {out}=n{nid}")
            nid += 1
    text = "\n".join(lines) + "\n"
    o = Oracle(text, lib)
    S = 33
    sp, tr = netgen.scenario_inputs(o.n_start, 3300, S)
    cfg = dp.config(grad_mode=0, tr_mode=2)
    d = dp.dp_design_load(ctx, text, lib)
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
    finally:
        dp.dp_design_free(d)
    check_lag1(o, g, sp, tr, range(S))


def test_lag1_with_independent_inputs_is_the_model(dp, ctx, small):
    """TR = 2P(1-P) at every startpoint: the lag-one mode gives Eq. 2 everywhere (tr_mode 1)."""
    text, o = small
    sp, _ = netgen.scenario_inputs(o.n_start, 3200, 16)
    tr = (2 * sp.astype(np.float64) * (1 - sp.astype(np.float64))).astype(np.float32)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        g2 = run_batch(dp, ctx, d, sp, tr, dp.config(grad_mode=0, tr_mode=2))
        g1 = run_batch(dp, ctx, d, sp, tr, dp.config(grad_mode=0, tr_mode=1))
    finally:
        dp.dp_design_free(d)
    np.testing.assert_array_equal(g2["sp"], g1["sp"])
    assert np.abs(g2["tr"] - g1["tr"]).max() <= 2e-6
    np.testing.assert_allclose(g2["power"], g1["power"], rtol=2e-6)


def test_lag1_mid_sampled(dp, ctx, library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["mid"])
    o = Oracle(text, library_text)
    S = 64
    sp, tr = netgen.scenario_inputs(o.n_start, 3400, S)
    cfg = dp.config(grad_mode=0, tr_mode=2)
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
        with pytest.raises(dp.DPError) as e:           # the single-scenario path has no lag-one mode
            dp.dp_set_inputs(ctx, d, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]), 1)
            dp.dp_propagate(ctx, d, cfg)
        assert e.value.name == "DP_EUNSUPPORTED"
    finally:
        dp.dp_design_free(d)
    check_lag1(o, g, sp, tr, [0, 31, 63])


def test_batch_only_startpoints_and_constants(dp, ctx, library_text):
    """Edge designs in the batched path: no cells at all, and constant cells only."""
    lib = "cell C0 Z 0.8 0\ncell C1 Z 1.6 1\n"
    only_start = "net a 1.0\nnet b 2.0\ninput a\ninput b\noutput a\noutput b\n"
    consts = "net a 1.0\ninput a\nnet y0 0.5\nnet y1 0.7\ncell u0 C0 Z=y0\ncell u1 C1 Z=y1\noutput y0\noutput y1\n"
    for text in (only_start, consts):
        o = Oracle(text, lib)
        S = 5
        sp, tr = netgen.scenario_inputs(o.n_start, 4400, S)
        for tr_mode in (0, 1, 2):
            cfg = dp.config(grad_mode=0, tr_mode=tr_mode)
            d = dp.dp_design_load(ctx, text, lib)
            try:
                g = run_batch(dp, ctx, d, sp, tr, cfg)
            finally:
                dp.dp_design_free(d)
            if tr_mode == 2:
                check_lag1(o, g, sp, tr, range(S))
            else:
                check_scenarios(o, g, sp, tr, cfg, range(S))


def test_batch_max_scenarios(dp, ctx, small):
    """The largest batch the tuner shapes for, 4,096 scenarios, on sampled scenarios."""
    text, o = small
    S = 4096
    sp, tr = netgen.scenario_inputs(o.n_start, 4500, S)
    cfg = dp.config(grad_mode=0, tr_mode=0)
    d = dp.dp_design_load(ctx, text, netgen.library_text())
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
    finally:
        dp.dp_design_free(d)
    check_scenarios(o, g, sp, tr, cfg, [0, 1, 2047, 4095])
