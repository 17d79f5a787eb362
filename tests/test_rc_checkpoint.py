"""Network checkpoints: round trip and corruption detection (CPU only)."""
import numpy as np
import pytest
import torch


def test_checkpoint_round_trip_and_checksum(tmp_path):
    from paper_1306_1373_gb300 import dctgb as D, rc
    net = D.Mlp(rc.init_params(3), act_bf16=True, device="cpu")
    net.m.normal_()
    net.v.uniform_()
    net.mean.fill_(0.5)
    net.std.fill_(2.0)
    net.c.step = 17
    p = tmp_path / "net.bin"
    rc.save(net, str(p), seed=3)
    back = rc.load(str(p), device="cpu")
    for a, b in ((net.params, back.params), (net.m, back.m), (net.v, back.v), (net.mean, back.mean),
                 (net.std, back.std)):
        assert torch.equal(a, b)
    assert back.step == 17 and back.c.act_bf16 == 1
    data = bytearray(p.read_bytes())
    data[100] ^= 0xFF
    p.write_bytes(bytes(data))
    with pytest.raises(ValueError):
        rc.load(str(p), device="cpu")


def test_init_params_layout_and_seed():
    from paper_1306_1373_gb300 import rc
    from oracle import mlp
    a = rc.init_params(5)
    assert a.shape == (9409,) and a.dtype == np.float32
    assert np.array_equal(a, rc.init_params(5)) and not np.array_equal(a, rc.init_params(6))
    assert np.allclose(a, mlp.init_params(5), atol=1e-7)   # same seeded draw as the oracle's initialiser


def test_autotune_cache_hit_skips_tuning(tmp_path, monkeypatch):
    """The cache stores the tuned shape under (GPU name, key, ops) and a
    later call with the same key prepares with it instead of re-tuning."""
    from paper_1306_1373_gb300 import dctgb as D
    calls = []
    monkeypatch.setattr(D, "dct_batch_prepare", lambda plan, items, ops, sse=None, shape=None, stream=None:
                        calls.append(("prepare", shape)))
    monkeypatch.setattr(D, "dct_autotune", lambda plan, stream=None: (calls.append(("tune",)) or
                                                                      ((128, 8, 32, 0), 0.5)))
    path = str(tmp_path / "tune.json")
    assert D.autotune_cached(None, None, 7, cache_path=path, key="grey8k") == (128, 8, 32, 0)
    assert calls == [("prepare", None), ("tune",)]
    calls.clear()
    assert D.autotune_cached(None, None, 7, cache_path=path, key="grey8k") == (128, 8, 32, 0)
    assert calls == [("prepare", (128, 8, 32, 0))]
    calls.clear()
    D.autotune_cached(None, None, 5, cache_path=path, key="grey8k")      # other ops: tuned again
    assert ("tune",) in calls
