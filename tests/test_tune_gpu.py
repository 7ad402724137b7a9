"""The tile tuner on the device: it measures both pass tiles through the C
ABI, writes a table, and a context applies it (only on the same device
model)."""
import json

import pytest
import torch

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_tuner_measures_and_context_applies(tmp_path):
    require_gpu()
    from paper_2107_01391_gb300 import binding, build, tune
    build.build()
    t = tune.table(tune.measure(sizes=(1 << 13, 1 << 15), reps=3))
    assert t["device_name"] == torch.cuda.get_device_name(0)
    assert t["narrow_max_n"] in (0, 1 << 13, 1 << 15)
    for shape in ("pairs", "keys"):
        for rec in t["measured"][shape].values():
            assert rec["wide_us"] > 0 and rec["narrow_us"] > 0
    path = tmp_path / "tune.json"
    path.write_text(json.dumps(dict(t, narrow_max_n=12345)))
    ctx = binding.Context(0)
    assert ctx.pass_tile_limit == 1 << 19
    assert ctx.apply_tuning(str(path))
    assert ctx.pass_tile_limit == 12345
    other = tmp_path / "other.json"
    other.write_text(json.dumps(dict(t, device_name="another GPU", narrow_max_n=7)))
    assert not ctx.apply_tuning(str(other))
    assert ctx.pass_tile_limit == 12345
    ctx.close()
