"""Shared test helpers: the per-variable scaled error of the parity gate and
tensor plumbing.  No method arithmetic here."""
import numpy as np


def scaled_err(a, b, g=None):
    """max over points and variables of |a-b| / max(|b|, S_v), S_v = max |b_v|
    over the (interior) grid; a, b shaped (nvars, ...)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if g is not None:
        a = a[..., g:-g, g:-g, g:-g]
        b = b[..., g:-g, g:-g, g:-g]
    nv = a.shape[0]
    A = a.reshape(nv, -1)
    B = b.reshape(nv, -1)
    S = np.abs(B).max(axis=1, keepdims=True)
    den = np.maximum(np.abs(B), S)
    den = np.where(den == 0, 1.0, den)
    return float((np.abs(A - B) / den).max())


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=torch.float64)


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
