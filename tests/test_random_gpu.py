"""Randomised sweep of the GPU path against the FP64 oracle: seeded random netlists over a
library with 0- to 4-input cells (constants, repeated and duplicated pins, DFF startpoints),
random inputs with degenerate values mixed in, and random configurations of every mode
(tr_mode, grad_mode, schedule, word count, one step or separate calls, host or device
buffers), then batched scenarios of random size in all three tr_modes.  Tolerances as in
test_parity_gpu.py and test_batch_gpu.py.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from tests.test_batch_gpu import check_lag1, check_scenarios, run_batch
from tests.test_parity_gpu import check_against_oracle, custom_case, gpu_run

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


def random_inputs(rng, n):
    sp = rng.uniform(0, 1, n).astype(np.float32)
    tr = (rng.uniform(0, 1, n) * 2 * np.minimum(sp, 1 - sp)).astype(np.float32)
    for _ in range(max(1, n // 20)):            # degenerate startpoints: constant, always toggling
        k = int(rng.integers(n))
        kind = int(rng.integers(4))
        if kind == 0:
            sp[k], tr[k] = 0.0, 0.0
        elif kind == 1:
            sp[k], tr[k] = 1.0, 0.0
        elif kind == 2:
            sp[k], tr[k] = 0.5, 1.0
        else:
            tr[k] = 0.0
    return sp, tr


@pytest.mark.parametrize("seed", range(48))
def test_random_single_scenario(dp, ctx, seed):
    rng = np.random.default_rng(9000 + seed)
    text, lib = custom_case(rng, n_in=int(rng.integers(4, 40)), n_cells=int(rng.integers(50, 1500)))
    o = Oracle(text, lib)
    sp, tr = random_inputs(rng, o.n_start)
    cfg = dp.config(tr_mode=int(rng.integers(2)), grad_mode=int(rng.integers(3)),
                    schedule=int(rng.choice([0, 1, 2, 3])), sim_words=int(rng.choice([4, 16, 20, 64, 100])),
                    seed=int(rng.integers(1 << 40)))
    use_step = bool(rng.integers(2))
    on_device = bool(rng.integers(2))
    g = gpu_run(dp, ctx, text, lib, sp, tr, cfg, use_step=use_step, on_device=on_device)
    check_against_oracle(o, g, sp, tr, cfg)


@pytest.mark.parametrize("seed", range(16))
def test_random_batched(dp, ctx, seed):
    rng = np.random.default_rng(9100 + seed)
    text, lib = custom_case(rng, n_in=int(rng.integers(4, 30)), n_cells=int(rng.integers(50, 800)))
    o = Oracle(text, lib)
    S = int(rng.integers(1, 300))
    sp = np.empty((o.n_start, S), np.float32)
    tr = np.empty((o.n_start, S), np.float32)
    for s in range(S):
        sp[:, s], tr[:, s] = random_inputs(rng, o.n_start)
    tr_mode = int(rng.integers(3))
    cfg = dp.config(grad_mode=0, tr_mode=tr_mode)
    d = dp.dp_design_load(ctx, text, lib)
    try:
        g = run_batch(dp, ctx, d, sp, tr, cfg)
    finally:
        dp.dp_design_free(d)
    scen = sorted({0, S - 1, *rng.integers(0, S, 4).tolist()})
    if tr_mode == 2:
        check_lag1(o, g, sp, tr, scen)
    else:
        check_scenarios(o, g, sp, tr, cfg, scen)
