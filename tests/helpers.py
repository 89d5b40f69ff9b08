"""Shared test helpers: the per-variable scaled error of the parity gate and
tensor plumbing.  No method arithmetic here."""
import numpy as np


class ParityErr(float):
    """The gate's value (a float) that also carries the secondary report: the
    raw pointwise relative error |a-b|/|b| over the points where
    |b| > 1e-3 S_v.  Its repr shows both, so a failing assertion prints them."""

    raw = None

    def __repr__(self):
        return "%.3e (raw pointwise rel. where |b| > 1e-3 S_v: %s)" % (
            float(self), "n/a" if self.raw is None else "%.3e" % self.raw)


def scaled_err(a, b, g=None):
    """max over points and variables of |a-b| / max(|b|, S_v), S_v = max |b_v|
    over the (interior) grid; a, b shaped (nvars, ...).  Since S_v bounds
    |b_v|, this is the per-variable max-normalised absolute error.  The
    returned ParityErr also carries the raw relative error where
    |b| > 1e-3 S_v (reported, not gated)."""
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
    out = ParityErr(float((np.abs(A - B) / den).max()))
    big = (np.abs(B) > 1e-3 * S) & (S > 0)
    if big.any():
        out.raw = float((np.abs(A - B)[big] / np.abs(B)[big]).max())
    return out


def to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=torch.float64)


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
