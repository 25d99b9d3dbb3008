"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def assert_elementwise(got, ref, scale, tol, what=""):
    """|got - ref| <= tol * scale for every element.

    ``scale`` bounds the magnitude of the terms each element sums, e.g. (|K| |V|)_ij
    for W = K V: the rounding of a product in any precision is a fraction of that sum
    of magnitudes, while a localized fault (a missed block, a wrong ragged edge) moves
    its elements by a whole term or more.  The message names the worst element."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    assert got.shape == ref.shape == scale.shape, (got.shape, ref.shape, scale.shape)
    bound = tol * scale + 1e-300
    err = np.abs(got - ref)
    ok = err <= bound
    if not ok.all():
        ratio = np.where(np.isfinite(err), err / bound, np.inf)
        i = np.unravel_index(int(np.argmax(ratio)), err.shape)
        raise AssertionError("%s: %d of %d elements beyond %.3g x scale; worst %s: got %r ref %r scale %r (%.3g x)"
                             % (what or "elementwise", int((~ok).sum()), ok.size, tol, i, got[i], ref[i],
                                scale[i], ratio[i]))


def product_scale(M, V):
    """Elementwise magnitude bound |M| |V| of the product M V (dense M)."""
    return np.abs(np.asarray(M, dtype=np.float64)) @ np.abs(np.asarray(V, dtype=np.float64))
