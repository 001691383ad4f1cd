"""Shared helpers for the GPU parity tests (tolerances, device transfers)."""
import numpy as np

U = 2.0 ** -53


def componentwise_error(C, ref, absAB):
    """max |C - ref| / (|A||B|) over entries with a nonzero denominator."""
    C = np.asarray(C, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.asarray(absAB, np.float64)
    mask = d > 0
    if not mask.any():
        return 0.0
    return float(np.max(np.abs(C - ref)[mask] / d[mask]))


def assert_within_bound(C, ref, absAB, n, factor=2.0):
    """|C - ref| <= factor * n * 2^-53 * |A||B| componentwise (zero where |A||B| = 0)."""
    C = np.asarray(C, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.asarray(absAB, np.float64)
    bound = factor * n * U * d
    bad = np.abs(C - ref) > bound
    if bad.any():
        i, k = np.argwhere(bad)[0]
        raise AssertionError(f"{bad.sum()} entries outside {factor}*N*u*|A||B| (N={n}); first ({i},{k}): "
                             f"got {C[i, k]!r}, ref {ref[i, k]!r}, bound {bound[i, k]!r}")


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()
