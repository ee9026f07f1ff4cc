"""Shared helpers for the GPU parity tests (host-side marshalling only)."""

from __future__ import annotations

import numpy as np


def to_dev_agents(agents: dict) -> dict:
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
            for k, v in agents.items()}


def subset_agents(agents: dict, idx) -> dict:
    idx = np.asarray(idx)
    return {k: np.ascontiguousarray(v[..., idx]) for k, v in agents.items()}


def u32(t) -> np.ndarray:
    """Device int32 tensor -> host uint32 bit pattern."""
    return t.cpu().numpy().view(np.uint32)


def f32_bits(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gate_allowance(obs64: np.ndarray, p: np.ndarray, R: np.ndarray, r_d: np.ndarray,
                   rel: float = 4e-7) -> np.ndarray:
    """Number of obstacle pairs per agent whose FP64 clamped distance lies
    within rel * r_d of the detection radius: FP32 may decide their gate the
    other way, which changes W by 1/r_d per pair."""
    out = np.zeros(p.shape[1], dtype=np.int64)
    for i in range(p.shape[1]):
        if not np.isfinite(r_d[i]):
            continue
        d = np.sqrt(((obs64 - p[:, i:i + 1]) ** 2).sum(axis=0))
        out[i] = int(np.count_nonzero(np.abs(d - R[i] - r_d[i]) <= rel * r_d[i] + 1e-7))
    return out
