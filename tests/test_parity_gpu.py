"""GPU path vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (the bar the hot path is held to):
* SP and TR of every net: 1e-5 absolute;
* toggle and ones counts: bit-exact;
* gradients: |g - g*| <= 1e-4 max(|g*|, 1e-3 max|g*|) (relative, near-zero floor);
* total power (FP64 reduction on the GPU of binary32 terms): 1e-6 relative;
* beta: within 1e-4 relative wherever TR_model > 0 (both sides carry P(net=0) as its own
  probability, so TR_model keeps full relative accuracy), hybrid TR within 1e-5 absolute.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests import _gates as G
from tests._netlists import custom_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def grad_close(g, g_star):
    g, g_star = np.asarray(g, np.float64), np.asarray(g_star, np.float64)
    if g_star.size == 0:
        return True
    floor = 1e-3 * np.abs(g_star).max()
    bad = np.abs(g - g_star) > 1e-4 * np.maximum(np.abs(g_star), floor)
    if bad.any():
        i = np.argmax(np.abs(g - g_star) / np.maximum(np.abs(g_star), floor + 1e-300))
        print(f"worst at {i}: {g[i]} vs {g_star[i]}")
    return not bad.any()


def gpu_run(dp, ctx, text, lib, sp_in, tr_in, cfg, use_step=False, on_device=False):
    d = dp.dp_design_load(ctx, text, lib)
    try:
        info = dp.dp_design_info(d)
        ns, nc, nn = info.n_start, info.n_cells, info.n_nets
        out = {}
        if on_device:
            dev = torch.device("cuda")
            sp_t = torch.from_numpy(np.ascontiguousarray(sp_in, np.float32)).to(dev)
            tr_t = torch.from_numpy(np.ascontiguousarray(tr_in, np.float32)).to(dev)
            dp.dp_set_inputs(ctx, d, sp_t, tr_t, 1, 1)
            bufs = {k: torch.zeros(n, dtype=torch.float32, device=dev)
                    for k, n in [("grad_sp_in", ns), ("grad_tr_in", ns), ("grad_pincap", nc), ("grad_cload", nn)]}
        else:
            dp.dp_set_inputs(ctx, d, np.ascontiguousarray(sp_in, np.float32), np.ascontiguousarray(tr_in, np.float32))
            bufs = {k: np.zeros(n, np.float32)
                    for k, n in [("grad_sp_in", ns), ("grad_tr_in", ns), ("grad_pincap", nc), ("grad_cload", nn)]}
        od = 1 if on_device else 0
        if use_step:
            watts = np.zeros(2)
            dp.dp_step(ctx, d, cfg, bufs["grad_sp_in"], bufs["grad_tr_in"], bufs["grad_pincap"],
                       bufs["grad_cload"], watts, od)
            out["power_model"], out["power_hybrid"] = watts
        else:
            dp.dp_propagate(ctx, d, cfg)
            out["power_model"] = dp.dp_total_power(ctx, d, 0)
            dp.dp_simulate(ctx, d, cfg)
            out["power_hybrid"] = dp.dp_total_power(ctx, d, 1)
            dp.dp_backward(ctx, d, cfg, bufs["grad_sp_in"], bufs["grad_tr_in"], bufs["grad_pincap"],
                           bufs["grad_cload"], od)
        if on_device:
            torch.cuda.synchronize()
            for k, v in bufs.items():
                out[k] = v.cpu().numpy()
        else:
            out.update(bufs)
        for k, dt in [("sp", np.float32), ("tr", np.float32), ("beta", np.float32), ("tr_hyb", np.float32),
                      ("toggles", np.uint32), ("ones", np.uint32)]:
            out[k] = np.zeros(nn, dt)
        dp.dp_get_nets(ctx, d, out["sp"], out["tr"], out["beta"], out["tr_hyb"], out["toggles"], out["ones"])
        out["info"] = info
        return out
    finally:
        dp.dp_design_free(d)


def check_against_oracle(o, g, sp_in, tr_in, cfg):
    ref = o.step(sp_in, tr_in, seed=cfg.seed, T=cfg.sim_words, grad_mode=cfg.grad_mode, tr_mode=cfg.tr_mode,
                 vdd=cfg.vdd, fclk=cfg.fclk, beta_min=cfg.beta_min, beta_max=cfg.beta_max)
    assert np.abs(g["sp"] - ref["sp"]).max(initial=0) <= 1e-5
    assert np.abs(g["tr"] - ref["tr"]).max(initial=0) <= 1e-5
    np.testing.assert_array_equal(g["toggles"], ref["toggles"])
    np.testing.assert_array_equal(g["ones"], ref["ones"])
    assert np.abs(g["tr_hyb"] - ref["tr_hyb"]).max(initial=0) <= 1e-5
    pos = ref["tr"] > 0
    assert np.all(np.abs(g["beta"][pos] - ref["beta"][pos]) <= 1e-4 * ref["beta"][pos])
    assert g["power_model"] == pytest.approx(ref["power_model"], rel=1e-6, abs=1e-30)
    assert g["power_hybrid"] == pytest.approx(ref["power_hybrid"], rel=1e-6, abs=1e-30)
    for k in ["grad_sp_in", "grad_tr_in", "grad_pincap", "grad_cload"]:
        assert grad_close(g[k], ref[k]), k
    return ref


@pytest.mark.parametrize("schedule", [0, 1, 2, 3])
@pytest.mark.parametrize("grad_mode", [0, 1, 2])
@pytest.mark.parametrize("tr_mode", [0, 1])
def test_small_all_modes(dp, ctx, library_text, grad_mode, tr_mode, schedule):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config(grad_mode=grad_mode, tr_mode=tr_mode, schedule=schedule)
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


@pytest.mark.parametrize("grad_mode", [0, 1])
def test_paper_small_shape(dp, ctx, library_text, grad_mode):
    """The 13,000-cell, 70-level netlist of the paper-shaped timings, against the oracle."""
    text = netgen.netlist_text(netgen.WORKLOADS["paper_small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config(grad_mode=grad_mode)
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg, use_step=grad_mode == 1)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


@pytest.mark.parametrize("use_step,on_device", [(False, True), (True, False), (True, True)])
def test_mid_paths(dp, ctx, library_text, use_step, on_device):
    text = netgen.netlist_text(netgen.WORKLOADS["mid"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config()
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg, use_step, on_device)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


def test_roofline_full_size(dp, ctx, library_text):
    """The 2M-cell netlist in the configuration the benchmark times (dp_step, device buffers)."""
    text = netgen.netlist_text(netgen.WORKLOADS["roofline"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config()
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg, use_step=True, on_device=True)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


def test_roofline_fwd_bwd_model(dp, ctx, library_text):
    """The 2M-cell netlist through dp_propagate + dp_backward with the model gradient (grad_mode 0)
    on device buffers: the forward + reverse pass the benchmark times alone (first with the
    startpoint SP gradient only, as timed, then with every gradient output)."""
    text = netgen.netlist_text(netgen.WORKLOADS["roofline"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    sp, tr = np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0])
    cfg = dp.config(grad_mode=0)
    dev = torch.device("cuda")
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        info = dp.dp_design_info(d)
        ns, nc, nn = info.n_start, info.n_cells, info.n_nets
        dp.dp_set_inputs(ctx, d, torch.from_numpy(sp).to(dev), torch.from_numpy(tr).to(dev), 1, 1)
        g = {k: torch.zeros(n, device=dev) for k, n in
             [("grad_sp_in", ns), ("grad_tr_in", ns), ("grad_pincap", nc), ("grad_cload", nn)]}
        for _ in range(2):
            dp.dp_propagate(ctx, d, cfg)
            dp.dp_backward(ctx, d, cfg, g["grad_sp_in"], None, None, None, 1)
        torch.cuda.synchronize()
        only_sp = g["grad_sp_in"].cpu().numpy()
        p_model = dp.dp_total_power(ctx, d, 0)
        dp.dp_backward(ctx, d, cfg, g["grad_sp_in"], g["grad_tr_in"], g["grad_pincap"], g["grad_cload"], 1)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in g.items()}
        net_sp, net_tr = np.zeros(nn, np.float32), np.zeros(nn, np.float32)
        dp.dp_get_nets(ctx, d, net_sp, net_tr, None, None, None, None)
    finally:
        dp.dp_design_free(d)
    sp_ref, tr_ref = o.forward(sp, tr, 0)
    assert np.abs(net_sp - sp_ref).max() <= 1e-5
    assert np.abs(net_tr - tr_ref).max() <= 1e-5
    assert p_model == pytest.approx(o.power(tr_ref), rel=1e-6)
    ref = o.backward(sp, tr, None, 0, 0)
    np.testing.assert_array_equal(only_sp, out["grad_sp_in"])
    for k in ["grad_sp_in", "grad_tr_in", "grad_pincap", "grad_cload"]:
        assert grad_close(out[k], ref[k]), k


def test_mid_exact_hybrid_gradient(dp, ctx, library_text):
    """grad_mode 2 (exact gradient of the hybrid power with beta held fixed) on the 120K-cell
    netlist through dp_step with device buffers."""
    text = netgen.netlist_text(netgen.WORKLOADS["mid"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config(grad_mode=2)
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg, use_step=True, on_device=True)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


def test_flip_probabilities_below_the_draw_resolution(dp, ctx, library_text):
    """Startpoints whose p10 or p01 lies in (0, 2^-16) get a zero threshold (reading R7): their
    chains never flip that way, so a startpoint with both below never toggles and its beta is
    beta_min (TR_model > 0, TR_acc = 0).  A probability of exactly 2^-16 keeps threshold 1.  GPU
    and oracle agree bit for bit on the counts and on beta."""
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    sp, tr = sp[:, 0].copy(), tr[:, 0].copy()
    tiny = [(0.5, 1e-5),                     # p10 = p01 = 1e-5
            (1e-5, 1e-5),                    # initial state always 0, p01 = 5e-6
            (0.99999, 1e-5),                 # p10 = 5e-6, p01 = 0.5
            (0.5, 2.0 ** -16),               # p10 = p01 = 2^-16 exactly: threshold 1
            (0.5, np.nextafter(np.float32(2.0 ** -16), np.float32(0)))]   # just below: threshold 0
    for k, (a, b) in enumerate(tiny):
        sp[k], tr[k] = np.float32(a), np.float32(b)
    cfg = dp.config()
    g = gpu_run(dp, ctx, text, library_text, sp, tr, cfg)
    ref = check_against_oracle(o, g, sp, tr, cfg)
    nets = o.start_nets()
    for k in (0, 1, 4):
        assert ref["toggles"][nets[k]] == 0 and g["toggles"][nets[k]] == 0
        assert g["beta"][nets[k]] == pytest.approx(cfg.beta_min)


@pytest.mark.parametrize("other_schedule", [0, 1, 3])
def test_step_is_deterministic(dp, ctx, library_text, other_schedule):
    """Two runs, and the persistent and per-level schedules, agree bit for bit."""
    text = netgen.netlist_text(netgen.WORKLOADS["mid"])
    sp, tr = netgen.scenario_inputs(netgen.WORKLOADS["mid"].n_start, 1000)
    a = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], dp.config(), use_step=True)
    b = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], dp.config(schedule=other_schedule), use_step=True)
    for k in ["sp", "tr", "beta", "toggles", "grad_sp_in", "grad_pincap", "grad_cload", "grad_tr_in"]:
        np.testing.assert_array_equal(a[k], b[k])
    assert a["power_model"] == b["power_model"] and a["power_hybrid"] == b["power_hybrid"]


# Schedule 0 picks, per design, the single-block passes, the single-cluster passes or the
# grid-wide ones.  Single block: the reverse block keeps n_nets pairs (16 B), n_edges edge
# adjoints (4 B) and n_levels + 1 level bounds (4 B) in at most 224 KiB of shared memory, and a
# level holds at most 1,024 cells.  Single cluster (otherwise): 16 blocks, each level cut into 16
# contiguous chunks, each block holding its chunks' pairs and their fanout ranges' edge
# adjoints in 224 KiB, a chunk at most 512 cells.
SMEM_MAX = 224 * 1024
CLUSTER = 16


def block_state_bytes(info):
    return info.n_nets * 16 + info.n_edges * 4 + (info.n_levels + 1) * 4


def cluster_state_bytes(text, lib, info, dp):
    """Shared memory of the busiest cluster block's reverse pass: every level (level 0: the
    startpoints) cut into 16 contiguous chunks, block b holding chunk b's pairs and their fanout
    ranges' edge adjoints, plus three tables of n_levels + 1 entries."""
    c = dp.dp_compile(text, lib)
    v = dp.dp_compiled_view_get(c)
    fptr = np.asarray(v["fout_ptr"]).astype(np.int64)
    lp = np.asarray(v["lvl_ptr"]).astype(np.int64)
    dp.dp_compiled_free(c)
    ns, nn, L = info.n_start, info.n_nets, info.n_levels
    owner = np.zeros(nn, np.int64)
    held = np.zeros(CLUSTER, np.int64)
    for lo, hi in [(0, ns)] + [(ns + lp[l - 1], ns + lp[l]) for l in range(1, L + 1)]:
        if hi > lo:
            b = np.arange(hi - lo) // -(-(hi - lo) // CLUSTER)
            owner[lo:hi] = b
            held += np.bincount(b, minlength=CLUSTER)
    edges = np.bincount(owner, weights=np.diff(fptr), minlength=CLUSTER).max()
    return int(held.max()) * 16 + int(edges) * 4 + 3 * (L + 1) * 4


PASS_CASES = {
    # name: (netlist spec or None for the random 0..4-input netlist, expected passes)
    "small": (netgen.WORKLOADS["small"], "block"),
    "serve_5000": (netgen.WORKLOADS["serve_5000"], "block"),
    "near_limit": (netgen.NetlistSpec(8_800, 64, 512, 30, 16, 7), "block"),    # 99.5 % of the block's room
    "just_over": (netgen.NetlistSpec(9_000, 64, 512, 30, 16, 7), "cluster"),   # 101.9 %
    "wide_level": (netgen.NetlistSpec(3_000, 200, 100, 2, 16, 8), "cluster"),  # 1,500 cells a level
    "random_4input": (None, "block"),
    "random_4input_large": (12_000, "cluster"),                                # 0..4-input cells, constants
    "serve_20000": (netgen.WORKLOADS["serve_20000"], "cluster"),
    "paper_small": (netgen.WORKLOADS["paper_small"], "cluster"),
    "mid": (netgen.WORKLOADS["mid"], "cluster"),                                # 98 % of a block's room
    "serve_300000": (netgen.WORKLOADS["serve_300000"], "grid"),
}


@pytest.mark.parametrize("case", list(PASS_CASES))
def test_block_and_cluster_passes_match_grid_passes(dp, ctx, library_text, case):
    """Schedule 0 takes the single-block or single-cluster forward and reverse passes exactly when
    a design fits them, and gives the same bits as the grid-wide passes (schedule 2) in every
    gradient mode, through both entry points and both output kinds; some designs are also
    checked against the oracle."""
    spec, expect = PASS_CASES[case]
    if spec is None:
        text, lib = custom_case(np.random.default_rng(77), n_in=12, n_cells=900)
    elif isinstance(spec, int):
        text, lib = custom_case(np.random.default_rng(78), n_in=200, n_cells=spec)
    else:
        text, lib = netgen.netlist_text(spec), library_text
    d = dp.dp_design_load(ctx, text, lib)
    info = dp.dp_design_info(d)
    dp.dp_design_free(d)
    c = dp.dp_compile(text, lib)
    width = int(np.diff(np.asarray(dp.dp_compiled_view_get(c)["lvl_ptr"])).max())
    dp.dp_compiled_free(c)
    block = block_state_bytes(info) <= SMEM_MAX and width <= 1024
    cluster = not block and cluster_state_bytes(text, lib, info, dp) <= SMEM_MAX and -(-width // CLUSTER) <= 512
    got = "block" if info.block_threads > 0 else "cluster" if info.cluster_threads > 0 else "grid"
    assert got == expect == ("block" if block else "cluster" if cluster else "grid")
    if got == "block":
        assert 256 <= info.block_threads <= 1024 and info.block_threads % 32 == 0 and info.cluster_threads == 0
    if got == "cluster":
        assert 64 <= info.cluster_threads <= 512 and info.cluster_threads % 32 == 0
        assert info.cluster_threads >= -(-width // CLUSTER)
    if case == "near_limit":
        assert block_state_bytes(info) > 0.97 * SMEM_MAX
    if case == "mid":
        assert cluster_state_bytes(text, lib, info, dp) > 0.85 * SMEM_MAX
    sp, tr = netgen.scenario_inputs(info.n_start, 1000)
    combos = [(0, 1, False, False), (1, 0, True, False), (2, 1, False, True), (0, 0, True, True)]
    if case in ("mid", "serve_300000"):
        combos = combos[1:3]
    for grad_mode, tr_mode, use_step, on_device in combos:
        runs = [gpu_run(dp, ctx, text, lib, sp[:, 0], tr[:, 0],
                        dp.config(grad_mode=grad_mode, tr_mode=tr_mode, schedule=sch), use_step, on_device)
                for sch in (0, 2)]
        for k in ["sp", "tr", "beta", "tr_hyb", "toggles", "grad_sp_in", "grad_tr_in", "grad_pincap",
                  "grad_cload"]:
            np.testing.assert_array_equal(runs[0][k], runs[1][k], err_msg=k)
        assert runs[0]["power_model"] == runs[1]["power_model"]
        assert runs[0]["power_hybrid"] == runs[1]["power_hybrid"]
        if case in ("near_limit", "random_4input", "just_over", "paper_small", "random_4input_large"):
            cfg = dp.config(grad_mode=grad_mode, tr_mode=tr_mode)
            check_against_oracle(Oracle(text, lib), runs[0], sp[:, 0], tr[:, 0], cfg)


# ---------------------------------------------------------------- edge cases


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("T", [2, 12, 33, 64, 97, 128])
def test_wide_and_constant_cells_ragged_words(dp, ctx, seed, T):
    rng = np.random.default_rng(seed)
    text, lib = custom_case(rng)
    o = Oracle(text, lib)
    sp = rng.uniform(0, 1, o.n_start).astype(np.float32)
    sp[0], sp[1] = 0.0, 1.0                      # degenerate inputs
    tr = (rng.uniform(0, 1, o.n_start) * 2 * np.minimum(sp, 1 - sp)).astype(np.float32)
    tr[2] = 0.0
    for grad_mode in [0, 1, 2]:
        cfg = dp.config(sim_words=T, grad_mode=grad_mode, seed=seed * 7)
        g = gpu_run(dp, ctx, text, lib, sp, tr, cfg)
        check_against_oracle(o, g, sp, tr, cfg)


@pytest.mark.parametrize("T", [16, 64, 128])
def test_startpoint_chains_both_forms(dp, ctx, library_text, T):
    """The startpoint generator's two forms: warps whose thresholds are all below 2^16, and
    warps (two startpoints each) holding a probability of exactly 1 (SP = 1, or TR = 2 SP so
    that p10 = 1); toggles and ones of every startpoint equal the oracle's."""
    n = 997
    text = "".join(f"net i{i} 1.0\ninput i{i}\n" for i in range(n)) + "output i0\n"
    o = Oracle(text, library_text)
    rng = np.random.default_rng(T)
    sp = rng.uniform(0.01, 0.99, n).astype(np.float32)
    tr = (rng.uniform(0, 1, n) * 2 * np.minimum(sp, 1 - sp)).astype(np.float32)
    sp[40], tr[40] = 1.0, 0.0
    sp[301], tr[301] = np.float32(0.25), np.float32(0.5)
    sp[302], tr[302] = np.float32(0.75), np.float32(0.5)
    sp[996], tr[996] = 0.0, 0.0
    cfg = dp.config(sim_words=T, grad_mode=1, seed=11 + T)
    g = gpu_run(dp, ctx, text, library_text, sp, tr, cfg)
    check_against_oracle(o, g, sp, tr, cfg)


def test_blob_design_gives_the_same_bits(dp, ctx, library_text):
    """A design loaded from a compiled-netlist blob runs exactly as one compiled from text."""
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    c = dp.dp_compile(text, library_text)
    try:
        blob = dp.dp_compiled_save(c)
    finally:
        dp.dp_compiled_free(c)
    sp, tr = netgen.scenario_inputs(netgen.WORKLOADS["small"].n_start, 77, 1)
    sp, tr = np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0])
    cfg = dp.config()
    outs = []
    for load in (lambda: dp.dp_design_load(ctx, text, library_text), lambda: dp.dp_design_load_blob(ctx, blob)):
        d = load()
        try:
            info = dp.dp_design_info(d)
            dp.dp_set_inputs(ctx, d, sp, tr)
            g = {k: np.zeros(n, np.float32) for k, n in [("sp", info.n_start), ("tr", info.n_start),
                                                          ("pin", info.n_cells), ("cl", info.n_nets)]}
            w = np.zeros(2)
            dp.dp_step(ctx, d, cfg, g["sp"], g["tr"], g["pin"], g["cl"], w, 0)
            outs.append((g, w))
        finally:
            dp.dp_design_free(d)
    for k in outs[0][0]:
        np.testing.assert_array_equal(outs[0][0][k], outs[1][0][k])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    with pytest.raises(dp.DPError) as e:
        dp.dp_design_load_blob(ctx, blob[:-3])
    assert e.value.name == "DP_EPARSE"


def test_boolean_inputs_exact(dp, ctx, library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2, o.n_start)
    g = gpu_run(dp, ctx, text, library_text, bits.astype(np.float32), np.zeros(o.n_start, np.float32),
                dp.config(grad_mode=0))
    want = G.boolean_eval(text, list(bits.astype(np.int64)))
    np.testing.assert_array_equal(g["sp"], want.astype(np.float32))


def test_only_startpoints_and_empty(dp, ctx, library_text):
    text = "net a 1.5\nnet b 0.5\ninput a\ninput b\noutput a\n"
    o = Oracle(text, library_text)
    sp, tr = np.array([0.3, 0.6], np.float32), np.array([0.2, 0.1], np.float32)
    cfg = dp.config()
    g = gpu_run(dp, ctx, text, library_text, sp, tr, cfg)
    check_against_oracle(o, g, sp, tr, cfg)
    d = dp.dp_design_load(ctx, "", library_text)
    dp.dp_set_inputs(ctx, d, np.zeros(0, np.float32), np.zeros(0, np.float32))
    dp.dp_propagate(ctx, d, cfg)
    assert dp.dp_total_power(ctx, d, 0) == 0.0
    dp.dp_design_free(d)


def test_sizing_delta(dp, ctx, library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config(grad_mode=0)
    rng = np.random.default_rng(8)
    # deltas in several calls; the third outgrows the design's staging, the fourth reuses it
    deltas = []
    for m in (5, 15, 1500, 40):
        cells = rng.choice(o.n_cells, m, replace=False).astype(np.int32)
        deltas.append((cells, rng.choice([0.8, 1.6, 3.2], m).astype(np.float32)))
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        dp.dp_set_inputs(ctx, d, sp[:, 0].copy(), tr[:, 0].copy())
        sizes = []
        for cells, caps in deltas:
            dp.dp_set_pincap(ctx, d, cells, caps)
            sizes.append(dp.dp_design_info(d).device_bytes)
        assert sizes[0] == sizes[1] and sizes[2] > sizes[1] and sizes[3] == sizes[2]
        dp.dp_propagate(ctx, d, cfg)
        p = dp.dp_total_power(ctx, d, 0)
        gsp = np.zeros(o.n_start, np.float32)
        gpin = np.zeros(o.n_cells, np.float32)
        dp.dp_backward(ctx, d, cfg, gsp, None, gpin, None)
    finally:
        dp.dp_design_free(d)
    for cells, caps in deltas:
        for c, v in zip(cells, caps):
            o.set_pincap(int(c), float(v))
    rsp, rtr = o.forward(sp[:, 0], tr[:, 0])
    assert p == pytest.approx(o.power(rtr), rel=1e-6)
    ref = o.backward(sp[:, 0], tr[:, 0])
    assert grad_close(gsp, ref["grad_sp_in"]) and grad_close(gpin, ref["grad_pincap"])


def test_call_order_and_argument_errors(dp, ctx, library_text):
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        cfg = dp.config()
        with pytest.raises(dp.DPError) as e:
            dp.dp_propagate(ctx, d, cfg)
        assert e.value.name == "DP_ESTATE"
        ns = dp.dp_design_info(d).n_start
        bad = np.full(ns, 0.5, np.float32)
        bad[3] = 1.5
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_inputs(ctx, d, bad, np.zeros(ns, np.float32))
        assert e.value.name == "DP_EINVAL"
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_inputs(ctx, d, np.zeros(ns, np.float32), np.zeros(ns, np.float32), 0)
        assert e.value.name == "DP_EINVAL"
        # more than one scenario selects the batched path (tests/test_batch_gpu.py)
        dp.dp_set_inputs(ctx, d, np.zeros(2 * ns, np.float32), np.zeros(2 * ns, np.float32), 2)
        dp.dp_set_inputs(ctx, d, np.full(ns, 0.5, np.float32), np.zeros(ns, np.float32))
        with pytest.raises(dp.DPError) as e:
            dp.dp_simulate(ctx, d, cfg)
        assert e.value.name == "DP_ESTATE"
        for bad_cfg in [dp.config(sim_words=1), dp.config(grad_mode=3), dp.config(beta_min=0.0),
                        dp.config(vdd=-1.0), dp.config(schedule=4)]:
            with pytest.raises(dp.DPError) as e:
                dp.dp_propagate(ctx, d, bad_cfg)
            assert e.value.name == "DP_EINVAL"
        dp.dp_propagate(ctx, d, dp.config(grad_mode=0))
        with pytest.raises(dp.DPError) as e:
            dp.dp_backward(ctx, d, dp.config(grad_mode=1), np.zeros(ns, np.float32))
        assert e.value.name == "DP_ESTATE"
        with pytest.raises(dp.DPError) as e:
            dp.dp_set_pincap(ctx, d, np.array([10 ** 7], np.int32), np.array([1.0], np.float32))
        assert e.value.name == "DP_EINVAL"
    finally:
        dp.dp_design_free(d)


def test_bounded_wait_gives_up(dp, ctx, library_text):
    """A grid barrier whose last arrival never comes gives up after its limit: DP_ETIMEOUT,
    and the context keeps working (no GPU fault is involved)."""
    with pytest.raises(dp.DPError) as e:
        dp.dp_selftest_wait(ctx, 0.05)
    assert e.value.name == "DP_ETIMEOUT"
    dp.dp_sync(ctx)   # the error word was cleared
    text = netgen.netlist_text(netgen.WORKLOADS["small"])
    o = Oracle(text, library_text)
    sp, tr = netgen.scenario_inputs(o.n_start, 1000)
    cfg = dp.config()
    g = gpu_run(dp, ctx, text, library_text, sp[:, 0], tr[:, 0], cfg, use_step=True)
    check_against_oracle(o, g, sp[:, 0], tr[:, 0], cfg)


def test_injected_allocation_failure(dp):
    """DP_FAULT=alloc:N fails the N-th device allocation on the host side: the load reports
    DP_ENOMEM and the process keeps working."""
    import subprocess
    import sys
    code = (
        "import numpy as np, torch\n"
        "from paper_2608_03778_gb300 import dp, netgen\n"
        "lib = netgen.library_text(); text = netgen.netlist_text(netgen.WORKLOADS['small'])\n"
        "ctx = dp.dp_create(0, None)\n"
        "try:\n    dp.dp_design_load(ctx, text, lib); print('NOFAIL')\n"
        "except dp.DPError as e:\n    print(e.name)\n"
        "d = dp.dp_design_load(ctx, text, lib); dp.dp_design_free(d); print('RECOVERED')\n"
    )
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, DP_FAULT="alloc:5"), cwd=root,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "DP_ENOMEM" in r.stdout and "RECOVERED" in r.stdout
