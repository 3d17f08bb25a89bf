"""Autotuner on the GPU: the chosen launch shape is one of the candidates,
its timings are positive, and the batch's results do not depend on it."""
import pytest

from test_gpu_batch import _mixed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_tuner_choice_keeps_results(lib, tmp_path):
    from paper_2211_00645_gb300.tune import Tuner
    items, _ = _mixed(lib)
    b = lib.Batch(max_items=8)
    b.set(items)
    b.run()
    torch.cuda.synchronize()
    ref = [(None if it["zmip"] is None else it["zmip"].clone(), it["ymip"].clone()) for it in items]
    t = Tuner(str(tmp_path / "t.json"))
    e = t.tune(items, kchunks=(16, 64, 256), ctas=(2, 4), reps=2)
    assert (e["kchunk"], e["ctas_per_sm"]) in [(k, c) for k in (16, 64, 256) for c in (2, 4)]
    assert len(e["candidates"]) == 6 and all(v > 0 for v in e["candidates"].values())
    k, c = t.best(items, torch.cuda.get_device_properties(0).multi_processor_count)
    b.set(items, k)
    b.run(c)
    torch.cuda.synchronize()
    b.check()
    for it, (z, y) in zip(items, ref):
        if z is not None:
            assert torch.equal(it["zmip"], z)
        assert torch.equal(it["ymip"], y)
