"""The level-latency probe behind the benchmark's latency floor: every figure positive and
finite, a level of the skeleton (barrier + dependent L2 gathers + store) costs at least its
barrier, and an out-of-range level count is rejected before any GPU work."""
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_probe_latency():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_03778_gb300 import dp
    ctx = dp.dp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        r = dp.dp_probe_latency(ctx, 64)
        for k in ("barrier_us_256", "level_us_256", "barrier_us_512", "level_us_512", "l2_load_us"):
            assert math.isfinite(r[k]) and 0 < r[k] < 100, (k, r[k])
        assert r["grid_blocks"] == torch.cuda.get_device_properties(0).multi_processor_count
        with pytest.raises(dp.DPError) as e:
            dp.dp_probe_latency(ctx, 8)
        assert e.value.name == "DP_EINVAL"
        dp.dp_sync(ctx)
    finally:
        dp.dp_destroy(ctx)
