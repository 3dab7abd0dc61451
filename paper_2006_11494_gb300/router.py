"""Router model buffers: packing the learned router's parameters into the
device layout of include/aot.h (AOT_MLP_MODEL_BYTES), and the JSON file the
trained model is kept in.  Marshalling only; the network runs in libaot.so."""
from __future__ import annotations

import json
import os

import numpy as np

from . import MLP_MODEL_BYTES, MLP_PARAMS

SIZES = ((64, 8), (64,), (64, 64), (64,), (3, 64), (3,))
DEFAULT_MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "router_model.json")


def pack(params_flat, in_mean, in_std, out_mean, out_std, margin, device="cuda"):
    """Model buffer (uint8 CUDA tensor) from float parameters and norms;
    parameters are rounded to bfloat16 (nearest even) by torch's cast."""
    import torch
    buf = torch.zeros(MLP_MODEL_BYTES, dtype=torch.uint8)
    hdr = np.zeros(32, np.float32)
    hdr[0:8] = in_mean
    hdr[8:16] = in_std
    hdr[16:19] = out_mean
    hdr[20:23] = out_std
    hdr[24] = margin
    buf[:128] = torch.from_numpy(hdr.view(np.uint8).copy())
    p = torch.as_tensor(np.asarray(params_flat, np.float32)).to(torch.bfloat16)
    assert p.numel() == MLP_PARAMS
    buf[128:128 + 2 * MLP_PARAMS] = p.view(torch.uint8)
    return buf.to(device)


def unpack(buf):
    """(params float64 [4931], in_mean, in_std, out_mean, out_std, margin)."""
    import torch
    b = buf.detach().cpu()
    hdr = b[:128].numpy().view(np.float32)
    p = b[128:128 + 2 * MLP_PARAMS].view(torch.bfloat16).float().numpy().astype(np.float64)
    return p, hdr[0:8].copy(), hdr[8:16].copy(), hdr[16:19].copy(), hdr[20:23].copy(), float(hdr[24])


def save(path, params_flat, in_mean, in_std, out_mean, out_std, margin, meta=None):
    with open(path, "w") as f:
        json.dump({"params_bf16_values": [float(x) for x in params_flat],
                   "in_mean": [float(x) for x in in_mean], "in_std": [float(x) for x in in_std],
                   "out_mean": [float(x) for x in out_mean], "out_std": [float(x) for x in out_std],
                   "margin": float(margin), "meta": meta or {}}, f)


def load(path=DEFAULT_MODEL_PATH, device="cuda"):
    """Model buffer from a saved JSON model (None if the file is absent)."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return pack(d["params_bf16_values"], d["in_mean"], d["in_std"], d["out_mean"], d["out_std"],
                d["margin"], device)


def with_margin(buf, margin):
    """Copy of a model buffer with another routing margin."""
    import torch
    b = buf.clone()
    m = torch.tensor([margin], dtype=torch.float32).view(torch.uint8)
    b[96:100] = m.to(b.device)
    return b
