"""Host side of the learned router's model buffer (no GPU): the byte layout the
C ABI documents, bfloat16 rounding of the parameters against the oracle's
round-to-nearest-even, the margin patch, the JSON round trip and the
committed model file."""
import json

import numpy as np

from oracle import mlp
from paper_2006_11494_gb300 import MLP_MODEL_BYTES, MLP_PARAMS, router


def _model(seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.7, MLP_PARAMS)
    # values on and near bfloat16 rounding ties
    theta[:4] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 3.0e-39]
    return (theta, rng.normal(0, 1, 8), rng.uniform(0.5, 2, 8), rng.normal(0, 1, 3),
            rng.uniform(0.5, 2, 3), 2.5)


def test_layout_and_rounding():
    theta, im, isd, om, osd, margin = _model(1)
    buf = router.pack(theta, im, isd, om, osd, margin, device="cpu")
    assert buf.numel() == MLP_MODEL_BYTES == 10240 and MLP_PARAMS == 4931
    raw = buf.numpy()
    hdr = raw[:128].view(np.float32)
    assert np.array_equal(hdr[0:8], im.astype(np.float32))      # bytes 0..31
    assert np.array_equal(hdr[8:16], isd.astype(np.float32))    # bytes 32..63
    assert np.array_equal(hdr[16:19], om.astype(np.float32))    # bytes 64..75
    assert hdr[19] == 0 and np.all(hdr[23:24] == 0)             # the unused fourth output
    assert np.array_equal(hdr[20:23], osd.astype(np.float32))   # bytes 80..91
    assert hdr[24] == np.float32(margin) and np.all(hdr[25:] == 0)
    p, *_ = router.unpack(buf)
    assert np.array_equal(p, mlp.bf16(theta.astype(np.float32).astype(np.float64)))
    assert np.all(raw[128 + 2 * MLP_PARAMS:] == 0)


def test_margin_patch_touches_only_the_margin():
    buf = router.pack(*_model(2), device="cpu")
    b2 = router.with_margin(buf, -7.25)
    diff = np.nonzero(buf.numpy() != b2.numpy())[0]
    assert diff.min() >= 96 and diff.max() < 100
    assert router.unpack(b2)[5] == -7.25


def test_json_round_trip(tmp_path):
    theta, im, isd, om, osd, margin = _model(3)
    theta = mlp.bf16(theta)
    path = tmp_path / "model.json"
    router.save(str(path), theta, im, isd, om, osd, margin, meta={"note": "test"})
    a = router.pack(theta, im, isd, om, osd, margin, device="cpu")
    b = router.load(str(path), device="cpu")
    assert np.array_equal(a.numpy(), b.numpy())
    assert router.load(str(tmp_path / "absent.json"), device="cpu") is None


def test_committed_model_is_well_formed():
    with open(router.DEFAULT_MODEL_PATH) as f:
        d = json.load(f)
    p = np.asarray(d["params_bf16_values"], np.float64)
    assert p.shape == (MLP_PARAMS,) and np.all(np.isfinite(p))
    assert np.array_equal(p, mlp.bf16(p))  # stored values are bfloat16 values
    assert len(d["in_mean"]) == 8 and len(d["in_std"]) == 8 and min(d["in_std"]) > 0
    assert len(d["out_mean"]) == 3 and len(d["out_std"]) == 3 and min(d["out_std"]) > 0
    buf = router.load(device="cpu")
    assert buf is not None and buf.numel() == MLP_MODEL_BYTES
