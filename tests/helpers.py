"""Shared test helpers (comparison metrics, skip logic)."""
import numpy as np
import pytest


def rel_inf(got, ref):
    """Per-substrate infinity-norm relative error max|got-ref| / max|ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for s in range(ref.shape[0]):
        den = np.abs(ref[s]).max()
        num = np.abs(got[s] - ref[s]).max()
        out.append(num / den if den > 0 else num)
    return np.asarray(out)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for s in range(ref.shape[0]):
        den = np.linalg.norm(ref[s])
        out.append(np.linalg.norm(got[s] - ref[s]) / (den if den > 0 else 1.0))
    return np.asarray(out)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch
