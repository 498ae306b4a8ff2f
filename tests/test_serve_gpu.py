"""The request server: results against the FP64 oracle (new inputs and sizing deltas),
bitwise identical alone and in a mix of other requests, the plain one-at-a-time mode,
HBM-budget admission and request validation.

Tolerances as for the batched path: power 1e-6 relative, gradients
|g - g*| <= 1e-4 max(|g*|, 1e-3 max|g*|).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2608_03778_gb300 import netgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp as _dp
    return _dp


def grad_close(g, g_star):
    g, g_star = np.asarray(g, np.float64), np.asarray(g_star, np.float64)
    floor = 1e-3 * np.abs(g_star).max()
    bad = np.abs(g - g_star) > 1e-4 * np.maximum(np.abs(g_star), floor)
    if bad.any():
        i = np.argmax(np.abs(g - g_star) / np.maximum(np.abs(g_star), floor + 1e-300))
        print(f"worst at {i}: {g[i]} vs {g_star[i]}")
    return not bad.any()


DESIGNS = ["small", "serve_5000", "serve_20000"]


@pytest.fixture(scope="module")
def texts():
    return {k: netgen.netlist_text(netgen.WORKLOADS[k]) for k in DESIGNS}


class Job:
    """One request with its own host buffers."""

    def __init__(self, dp, design, ns, nc, sp=None, tr=None, cells=None, caps=None, grad=0):
        self.design, self.sp, self.tr, self.cells, self.caps, self.grad = design, sp, tr, cells, caps, grad
        self.power = np.zeros(1)
        self.gsp = np.zeros(ns, np.float32) if grad else None
        self.gtr = np.zeros(ns, np.float32) if grad else None
        self.gpin = np.zeros(nc, np.float32) if grad else None
        self.req = dp.request(design, self.power, sp, tr, cells, caps, grad, self.gsp, self.gtr, self.gpin)

    def result(self):
        return [self.power.copy()] + ([self.gsp.copy(), self.gtr.copy(), self.gpin.copy()] if self.grad else [])


def make_jobs(dp, ids, infos, n, seed, refs):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        k = int(rng.integers(len(ids)))
        ns, nc = infos[k].n_start, infos[k].n_cells
        grad = int(rng.integers(2))
        if rng.integers(2):
            sp, tr = netgen.scenario_inputs(ns, seed * 1000 + i, 1)
            jobs.append(Job(dp, ids[k], ns, nc, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]),
                            grad=grad))
        else:
            m = max(1, nc // 100)
            cells = rng.choice(nc, m, replace=False).astype(np.int32)
            caps = rng.choice(np.array([1.6, 3.2], np.float32), m)
            jobs.append(Job(dp, ids[k], ns, nc, cells=cells, caps=caps, grad=grad))
    return jobs


@pytest.fixture(scope="module")
def server(dp, texts):
    cfg = dp.server_config(max_batch=16)
    srv = dp.dp_server_create(cfg)
    lib = netgen.library_text()
    ids, infos, refs = [], [], []
    for k in DESIGNS:
        ns = netgen.WORKLOADS[k].n_start
        sp, tr = netgen.scenario_inputs(ns, 42, 1)
        ref = (np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]))
        ids.append(dp.dp_server_add_design(srv, texts[k], lib, *ref))
        infos.append(dp.dp_server_design_info(srv, ids[-1]))
        refs.append(ref)
    yield srv, ids, infos, refs
    dp.dp_server_destroy(srv)


def run(dp, srv, jobs, together=True):
    if together:
        tickets = [dp.dp_server_submit(srv, j.req) for j in jobs]
        return [dp.dp_server_wait(srv, t, 60.0) for t in tickets]
    return [dp.dp_server_wait(srv, dp.dp_server_submit(srv, j.req), 60.0) for j in jobs]


def test_server_matches_oracle(dp, server, texts):
    srv, ids, infos, refs = server
    lib = netgen.library_text()
    jobs = make_jobs(dp, ids, infos, 24, 7, refs)
    for j in jobs:
        j.grad = 1
        ns, nc = infos[ids.index(j.design)].n_start, infos[ids.index(j.design)].n_cells
        j.gsp, j.gtr, j.gpin = np.zeros(ns, np.float32), np.zeros(ns, np.float32), np.zeros(nc, np.float32)
        j.req = dp.request(j.design, j.power, j.sp, j.tr, j.cells, j.caps, 1, j.gsp, j.gtr, j.gpin)
    run(dp, srv, jobs)
    for j in jobs:
        k = ids.index(j.design)
        o = Oracle(texts[DESIGNS[k]], lib)
        sp, tr = (j.sp, j.tr) if j.sp is not None else refs[k]
        if j.cells is not None:
            for c, cap in zip(j.cells, j.caps):
                o.set_pincap(int(c), float(cap))
        _, trf = o.forward(sp, tr, 0)
        assert j.power[0] == pytest.approx(o.power(trf), rel=1e-6)
        ref = o.backward(sp, tr, None, 0, 0)
        assert grad_close(j.gsp, ref["grad_sp_in"])
        assert grad_close(j.gtr, ref["grad_tr_in"])
        assert grad_close(j.gpin, ref["grad_pincap"])


def test_alone_equals_in_mix(dp, server):
    srv, ids, infos, refs = server
    probe = make_jobs(dp, ids, infos, 6, 11, refs)
    for j in probe:
        j.grad = 1
        ns, nc = infos[ids.index(j.design)].n_start, infos[ids.index(j.design)].n_cells
        j.gsp, j.gtr, j.gpin = np.zeros(ns, np.float32), np.zeros(ns, np.float32), np.zeros(nc, np.float32)
        j.req = dp.request(j.design, j.power, j.sp, j.tr, j.cells, j.caps, 1, j.gsp, j.gtr, j.gpin)
    run(dp, srv, probe, together=False)                # each alone
    alone = [j.result() for j in probe]
    for j in probe:
        for a in j.result():
            a[...] = 0
    mix = make_jobs(dp, ids, infos, 90, 12, refs)
    order = mix[:30] + probe[:3] + mix[30:60] + probe[3:] + mix[60:]
    run(dp, srv, order)                                # in a mix, batched with others
    st = dp.dp_server_get_stats(srv)
    assert st.max_batch_seen > 1
    for j, a in zip(probe, alone):
        for x, y in zip(j.result(), a):
            np.testing.assert_array_equal(x, y)


def test_burst_submission_gives_the_same_bits(dp, server):
    """dp_server_submit_many queues a burst in one step: the results equal those of the same
    requests run one at a time, the batches are full, and one invalid request in a burst
    queues nothing."""
    srv, ids, infos, refs = server
    jobs = make_jobs(dp, ids, infos, 60, 21, refs)
    run(dp, srv, jobs, together=False)
    alone = [j.result() for j in jobs]
    for j in jobs:
        for a in j.result():
            a[...] = 0
    st0 = dp.dp_server_get_stats(srv)
    tickets = dp.dp_server_submit_many(srv, [j.req for j in jobs])
    assert len(tickets) == len(jobs) and len(set(tickets)) == len(jobs)
    for t in tickets:
        dp.dp_server_wait(srv, t, 60.0)
    st1 = dp.dp_server_get_stats(srv)
    assert st1.requests - st0.requests == len(jobs)
    assert (st1.requests - st0.requests) / (st1.batches - st0.batches) > 4   # 60 requests on 3 designs, max 16
    for j, a in zip(jobs, alone):
        for x, y in zip(j.result(), a):
            np.testing.assert_array_equal(x, y)
    bad = dp.request(99, np.zeros(1))
    with pytest.raises(dp.DPError) as e:
        dp.dp_server_submit_many(srv, [jobs[0].req, bad])
    assert e.value.name == "DP_EINVAL"
    st2 = dp.dp_server_get_stats(srv)
    assert st2.requests == st1.requests   # nothing from the rejected burst was queued or run
    assert dp.dp_server_submit_many(srv, []) == []


def test_reference_batches_skip_the_forward_with_the_same_bits(dp, server):
    """A batch of requests that all use the reference inputs starts from the forward state
    cached when the design was added; the same requests with the reference inputs given
    explicitly run the forward pass.  Both give the same bits (sizing deltas and gradients
    included)."""
    srv, ids, infos, refs = server
    rng = np.random.default_rng(31)
    implicit, explicit = [], []
    for i in range(12):
        k = i % len(ids)
        ns, nc = infos[k].n_start, infos[k].n_cells
        m = max(1, nc // 50)
        cells = rng.choice(nc, m, replace=False).astype(np.int32)
        caps = rng.choice(np.array([1.6, 3.2], np.float32), m)
        implicit.append(Job(dp, ids[k], ns, nc, cells=cells, caps=caps, grad=1))
        explicit.append(Job(dp, ids[k], ns, nc, refs[k][0], refs[k][1], cells=cells, caps=caps, grad=1))
    run(dp, srv, implicit)   # batches of reference-input requests only
    run(dp, srv, explicit)
    for a, b in zip(implicit, explicit):
        for x, y in zip(a.result(), b.result()):
            np.testing.assert_array_equal(x, y)


def test_plain_mode_gives_the_same_bits(dp, server, texts):
    srv, ids, infos, refs = server
    jobs = make_jobs(dp, ids, infos, 12, 21, refs)
    run(dp, srv, jobs)
    batched = [j.result() for j in jobs]
    plain = dp.dp_server_create(dp.server_config(plain=1))
    try:
        lib = netgen.library_text()
        pids = [dp.dp_server_add_design(plain, texts[k], lib, *refs[i]) for i, k in enumerate(DESIGNS)]
        assert pids == ids
        for j in jobs:
            for a in j.result():
                a[...] = 0
        lat = run(dp, plain, jobs, together=False)
        assert all(x > 0 for x in lat)
        assert dp.dp_server_get_stats(plain).max_batch_seen == 1
    finally:
        dp.dp_server_destroy(plain)
    for j, b in zip(jobs, batched):
        for x, y in zip(j.result(), b):
            np.testing.assert_array_equal(x, y)


def test_two_slots_per_design_give_the_same_bits(dp, server, texts):
    """Two batch slots per design (two copies of its device state, batches of one design
    overlapping): every result bitwise equal to the one-slot server's."""
    srv1, ids, infos, refs = server
    srv2 = dp.dp_server_create(dp.server_config(max_batch=16, slots_per_design=2))
    try:
        lib = netgen.library_text()
        for k, ref in zip(DESIGNS, refs):
            dp.dp_server_add_design(srv2, texts[k], lib, *ref)
        st = dp.dp_server_get_stats(srv2)
        assert st.designs == len(DESIGNS)
        info2 = dp.dp_server_design_info(srv2, ids[0])
        assert info2.device_bytes > infos[0].device_bytes
        jobs = make_jobs(dp, ids, infos, 120, 77, refs)
        run(dp, srv2, jobs)
        two = [j.result() for j in jobs]
        run(dp, srv1, jobs, together=False)
        for a, b in zip(two, [j.result() for j in jobs]):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
    finally:
        dp.dp_server_destroy(srv2)
    with pytest.raises(dp.DPError):
        dp.dp_server_create(dp.server_config(slots_per_design=9))


def test_budget_admission_and_errors(dp, texts):
    lib = netgen.library_text()
    srv = dp.dp_server_create(dp.server_config(max_batch=8, hbm_budget=32 << 20))
    try:
        i = dp.dp_server_add_design(srv, texts["small"], lib)
        with pytest.raises(dp.DPError) as e:
            dp.dp_server_add_design(srv, netgen.netlist_text(netgen.WORKLOADS["mid"]), lib)
        assert e.value.name == "DP_ENOMEM"
        st = dp.dp_server_get_stats(srv)
        assert st.designs == 1 and 0 < st.device_bytes <= 32 << 20
        info = dp.dp_server_design_info(srv, i)
        power = np.zeros(1)
        for bad in [dict(design=5), dict(cells=np.array([10 ** 6], np.int32), pincap=np.ones(1, np.float32)),
                    dict(sp=np.full(info.n_start, 2.0, np.float32), tr=np.zeros(info.n_start, np.float32)),
                    dict(sp=np.full(info.n_start, 0.5, np.float32))]:
            kw = dict(design=i)
            kw.update(bad)
            with pytest.raises(dp.DPError) as e:
                dp.dp_server_submit(srv, dp.request(power=power, **kw))
            assert e.value.name == "DP_EINVAL"
        t = dp.dp_server_submit(srv, dp.request(i, power))      # reference inputs, design caps
        assert dp.dp_server_wait(srv, t, 60.0) > 0
        assert power[0] > 0
        with pytest.raises(dp.DPError) as e:
            dp.dp_server_wait(srv, t)                            # released
        assert e.value.name == "DP_EINVAL"
    finally:
        dp.dp_server_destroy(srv)
    with pytest.raises(dp.DPError):
        dp.dp_server_create(dp.server_config(max_batch=0))


def test_sizing_deltas_beyond_the_reserved_capacity(dp, texts):
    """Batches whose sizing deltas outgrow the entries reserved at admission (the arrays grow
    in stream order), with requests without deltas and cells listed twice in between: results
    match the oracle and the plain loop bit for bit."""
    lib = netgen.library_text()
    text = texts["small"]
    ns = netgen.WORKLOADS["small"].n_start
    sp, tr = netgen.scenario_inputs(ns, 42, 1)
    ref = (np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]))
    srv = dp.dp_server_create(dp.server_config(max_batch=4))
    plain = dp.dp_server_create(dp.server_config(plain=1))
    try:
        i = dp.dp_server_add_design(srv, text, lib, *ref)
        assert dp.dp_server_add_design(plain, text, lib, *ref) == i
        nc = dp.dp_server_design_info(srv, i).n_cells
        rng = np.random.default_rng(5)
        jobs = []
        for r in range(8):
            if r % 3 == 1:
                jobs.append(Job(dp, i, ns, nc, grad=1))                   # no delta
                continue
            cells = np.concatenate([rng.permutation(nc), rng.permutation(nc)]).astype(np.int32)
            caps = rng.choice(np.array([0.8, 1.6, 3.2], np.float32), cells.size)
            jobs.append(Job(dp, i, ns, nc, cells=cells, caps=caps, grad=1))   # 2 entries per cell
        run(dp, srv, jobs)
        assert dp.dp_server_get_stats(srv).max_batch_seen > 1
        served = [j.result() for j in jobs]
        run(dp, plain, jobs, together=False)
        for j, a in zip(jobs, served):
            for x, y in zip(j.result(), a):
                np.testing.assert_array_equal(x, y)
        for j in jobs[:3]:
            o = Oracle(text, lib)
            if j.cells is not None:
                for c, cap in zip(j.cells, j.caps):   # the last entry of a cell counts
                    o.set_pincap(int(c), float(cap))
            _, trf = o.forward(*ref, 0)
            assert j.power[0] == pytest.approx(o.power(trf), rel=1e-6)
            g = o.backward(*ref, None, 0, 0)
            assert grad_close(j.gsp, g["grad_sp_in"]) and grad_close(j.gpin, g["grad_pincap"])
    finally:
        dp.dp_server_destroy(srv)
        dp.dp_server_destroy(plain)
