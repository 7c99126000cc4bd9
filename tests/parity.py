"""Shared helpers for the GPU-vs-oracle parity tests."""
import numpy as np


def rel_err(got, ref, floor=1e-3):
    """Per-tensor infinity-norm error relative to the reference's scale."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), floor))


def to_np(t):
    return t.detach().cpu().numpy()


def upstream(rng, H, W, mask=None):
    """Seeded random upstream gradients for the 12 rendered channels; zero on `mask`-False pixels."""
    dr = rng.standard_normal((3, H, W))
    df = rng.standard_normal((8, H, W))
    du = rng.standard_normal((H, W))
    if mask is not None:
        dr[:, ~mask] = 0
        df[:, ~mask] = 0
        du[~mask] = 0
    return dr, df, du
