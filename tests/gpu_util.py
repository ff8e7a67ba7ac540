"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import torch


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def pack_mask(mask):
    """uint8/bool H x W -> uint32 words, ceil(W/32) per row, pixel (i, j) at bit j % 32."""
    m = np.asarray(mask, dtype=bool)
    H, W = m.shape
    nw = (W + 31) // 32
    pad = np.zeros((H, nw * 32), dtype=np.uint64)
    pad[:, :W] = m
    bits = pad.reshape(H, nw, 32) << np.arange(32, dtype=np.uint64)
    return bits.sum(axis=2).astype(np.uint32)


def rel_close(a, b, rtol, atol=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) <= atol + rtol * np.maximum(np.abs(a), np.abs(b))


def float_ulp(x):
    return np.spacing(np.abs(np.asarray(x, dtype=np.float32))).astype(np.float64)
