"""dp_power_noalloc: the power reduction for callers that cannot allocate device memory (a host
framework that owns every device byte through its own pool, or a service that plans its memory
ahead and must not let a cudaMalloc synchronise the device).  Its scratch is a fixed array in the
library's device memory.  Checked through the C-ABI on two calls in a row, within the power
tolerance of the other GPU tests (1e-6 relative), against dp_total_power on the same nets and
against the FP64 oracle's power (Eq. 1) of the oracle's own TR and beta; device free memory must
not change across calls after the first, and an error the caller left pending must survive a call.

This file is collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen
from tests import _gates as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def cload_user(text, library_text):
    """C_load per net in declaration order, from the netlist text (Eq. 1 loads)."""
    nets, wire, inputs, dffs, cells = G.parse_netlist(text)
    caps = {}
    for line in library_text.splitlines():
        f = line.split()
        if f and f[0] == "cell":
            caps[f[1]] = (f[2], float(f[3]))
        elif f and f[0] == "seq":
            caps[f[1]] = (None, float(f[4]))
    c = np.array(wire, np.float64)
    for d, _ in dffs:
        c[d] += caps["DFF_X1"][1]
    for ref, pins in cells:
        out, pc = caps[ref]
        for p, n in pins.items():
            if p != out:
                c[n] += pc
    return c.astype(np.float32)


@pytest.mark.parametrize("name", ["small", "mid"])
def test_noalloc_power_matches_total_power(name, library_text):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp
    text = netgen.netlist_text(netgen.WORKLOADS[name])
    stream = torch.cuda.current_stream().cuda_stream
    ctx = dp.dp_create(0, stream)
    d = dp.dp_design_load(ctx, text, library_text)
    try:
        info = dp.dp_design_info(d)
        nn = info.n_nets
        sp, tr = netgen.scenario_inputs(info.n_start, 1000)
        cfg = dp.config()
        dp.dp_set_inputs(ctx, d, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]))
        dp.dp_propagate(ctx, d, cfg)
        dp.dp_simulate(ctx, d, cfg)
        want_model = dp.dp_total_power(ctx, d, 0)
        want_hyb = dp.dp_total_power(ctx, d, 1)
        dev = torch.device("cuda", 0)
        tr_d = torch.zeros(nn, device=dev)
        beta_d = torch.zeros(nn, device=dev)
        dp.dp_get_nets(ctx, d, None, tr_d, beta_d, None, None, None, 1)
        cl_d = torch.from_numpy(cload_user(text, library_text)).to(dev)
        watts = torch.zeros(2, dtype=torch.float64, device=dev)
        # the oracle's powers (Eq. 1) from its own forward pass, simulation and beta
        o = Oracle(text, library_text)
        ref = o.step(np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]), seed=cfg.seed,
                     T=cfg.sim_words, grad_mode=0)
        np.testing.assert_allclose(cl_d.cpu().numpy(), o.cload(), rtol=1e-6)
        free_after_first = None
        for i in range(4):   # calls in a row share the scratch
            watts.fill_(-1.0)
            dp.dp_power_noalloc(0, tr_d, None, cl_d, nn, cfg.vdd, cfg.fclk, watts[0:1], stream)
            dp.dp_power_noalloc(0, tr_d, beta_d, cl_d, nn, cfg.vdd, cfg.fclk, watts[1:2], stream)
            torch.cuda.synchronize()
            got = watts.cpu().numpy()
            assert got[0] == pytest.approx(want_model, rel=1e-6)
            assert got[1] == pytest.approx(want_hyb, rel=1e-6)
            assert got[0] == pytest.approx(ref["power_model"], rel=1e-6)
            assert got[1] == pytest.approx(ref["power_hybrid"], rel=1e-6)
            # after the first call (which may load the kernels' code) no call takes device memory
            free = torch.cuda.mem_get_info(0)[0]
            if free_after_first is None:
                free_after_first = free
            assert free == free_after_first
    finally:
        dp.dp_design_free(d)
        dp.dp_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, device="cuda")
    with pytest.raises(dp.DPError) as e:
        dp.dp_power_noalloc(0, x, None, x, 33_554_432 + 1, 0.8, 1e9, w)
    assert e.value.name == "DP_EUNSUPPORTED"
    with pytest.raises(dp.DPError) as e:
        dp.dp_power_noalloc(0, None, None, x, 4, 0.8, 1e9, w)
    assert e.value.name == "DP_EINVAL"
    dp.dp_power_noalloc(0, x, None, x, 0, 0.8, 1e9, w)   # empty: writes 0
    torch.cuda.synchronize()
    assert w.item() == 0.0


def test_noalloc_leaves_a_pending_error_alone():
    """An error the caller left pending on this thread (a launch the runtime rejected on the host;
    nothing reached the GPU) is neither this call's result nor cleared by it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.ones(1000, device="cuda")
    dp.dp_selftest_pending_error(2)
    code = dp.dp_selftest_pending_error(1)
    try:
        assert code != 0
        dp.dp_power_noalloc(0, x, None, x, 1000, 0.8, 1e9, w)   # must not raise
        torch.cuda.synchronize()
        assert w.item() == pytest.approx(0.5 * 0.8 * 0.8 * 1e9 * 1e-15 * 1000, rel=1e-12)
        assert dp.dp_selftest_pending_error(0) == code
    finally:
        dp.dp_selftest_pending_error(2)
    assert dp.dp_selftest_pending_error(0) == 0
