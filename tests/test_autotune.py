"""Autotuner: cache keys, cache round trip (CPU) and tuned shapes that keep the
results bit-exact (GPU)."""
import numpy as np
import pytest


def test_cache_key_buckets():
    from paper_2308_13289_b300 import autotune
    assert autotune.cache_key("B300", 100, 1024, 100000) == autotune.cache_key("B300", 100, 1000, 70000)
    assert autotune.cache_key("B300", 100, 1024, 1e5) != autotune.cache_key("B300", 250, 1024, 1e5)
    assert autotune.cache_key("B300", 100, 1024, 1e5) != autotune.cache_key("B300", 100, 8192, 1e5)


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_2308_13289_b300 import autotune
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    assert autotune.load_cache() == {}
    autotune.save_cache({"k": {"warps": 4, "chunk": 64, "ms": 1.0, "table": []}})
    assert autotune.load_cache()["k"]["warps"] == 4


@pytest.mark.gpu
def test_tuned_shape_is_bit_exact(tmp_path, monkeypatch):
    import torch

    import lobgen
    import paper_2308_13289_b300 as eng
    from engine_harness import assert_same, gpu_outputs
    from paper_2308_13289_b300 import autotune
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    m, off = lobgen.generate(lobgen.make_params(3), [2000] * 64)
    d, o = eng.messages_to_device(m), torch.from_numpy(off).cuda()
    shape = autotune.tune(64, 100, d, o, reps=1, warps=(1, 4, 8), chunks=(32, 128))
    assert not shape["cached"] and len(shape["table"]) == 6
    again = autotune.tune(64, 100, d, o)
    assert again["cached"] and again["warps"] == shape["warps"]
    a = eng.Engine(64, 100, 2048)
    a.process_batch(d, o)
    b = eng.Engine(64, 100, 2048)
    autotune.apply(b, shape)
    b.process_batch(d, o)
    assert_same(gpu_outputs(b), gpu_outputs(a))
