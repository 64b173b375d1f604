"""Error measures of the GPU tests: relative 2-norm, element-wise maximum, and
the normalisation of the paper's a-priori bound (Sec. 3, eq. (KERR_estimate):
the largest error divided by ||x||_1 K(0))."""
import numpy as np


def _np(a):
    """numpy FP64 copy of an array or a (CUDA or CPU) torch tensor."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def rel(a, b):
    a, b = _np(a), _np(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def errors(y, ref, x=None, k0=1.0):
    """dict(rel2, relmax, kerr): ||e||_2/||ref||_2, max|e|/max|ref|, max|e|/(||x||_1 K(0))."""
    y, ref = _np(y), _np(ref)
    e = np.abs(y - ref)
    out = {"rel2": rel(y, ref), "relmax": float(e.max() / np.abs(ref).max())}
    if x is not None:
        out["kerr"] = float(e.max() / (np.abs(_np(x)).sum() * k0))
    return out


def assert_close(y, ref, tol, x=None, k0=1.0, what=""):
    """The 2-norm within tol, and every element within 3 tol of the largest reference
    value (so one wrong node cannot hide in the 2-norm); with x, the paper's
    normalisation max|e| / (||x||_1 K(0)) within tol as well."""
    err = errors(y, ref, x, k0)
    assert err["rel2"] < tol, (what, err)
    assert err["relmax"] < 3.0 * tol, (what, err)
    if x is not None:
        assert err["kerr"] < tol, (what, err)
    return err
