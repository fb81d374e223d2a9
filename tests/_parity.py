"""Comparison of a GPU result with the FP64 oracle's, shared by the GPU tests.

x from the FP32 kernel must be within `tol` of the oracle's x in two senses:
the relative L2 error ||x_gpu - x_o|| / ||x_o||, and every element,
max_j |x_gpu,j - x_o,j| <= tol * ||x_o||_inf.  The second catches an error
confined to a few columns (the tail slice, one CTA's slice of the average)
that the L2 norm of a long vector would hide.  Non-finite GPU values fail."""
import numpy as np


def assert_close(x_gpu, x_o, tol, what=""):
    xg = np.asarray(x_gpu, np.float64).ravel()
    xo = np.asarray(x_o, np.float64).ravel()
    assert xg.shape == xo.shape, (what, xg.shape, xo.shape)
    assert np.all(np.isfinite(xg)), f"{what}: non-finite GPU values"
    if xo.size == 0:
        return 0.0
    diff = np.abs(xg - xo)
    ref2 = np.linalg.norm(xo)
    refi = np.max(np.abs(xo))
    rel = np.linalg.norm(diff) / max(ref2, 1e-300)
    worst = np.max(diff) / max(refi, 1e-300)
    j = int(np.argmax(diff))
    assert rel < tol, f"{what}: relative L2 error {rel:.3e} >= {tol:g}"
    assert worst <= tol, (f"{what}: element {j} differs by {diff[j]:.3e} "
                          f"({worst:.3e} of max|x_o| = {refi:.3e}), above {tol:g}")
    return rel
