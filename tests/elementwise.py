"""Element-wise comparison of a device result with its oracle reference.

Each row (a camera's 9 parameters, a point's 3, one camera's 9 entries of b') and each 9 x 9 camera block of
a cluster system is compared on its own: the largest difference in the row or block over the largest
reference value in it.  One wrong camera, point or block therefore cannot hide under the norm of the rest.
A reference row or block that is exactly zero (two cameras of a cluster that share no point) must come back
exactly zero, unless `floor` > 0, which lets the scale of a row fall no lower than `floor` times the largest
reference value overall (for quantities whose small rows carry the absolute error of the large ones).

`cols` scales each element by the largest reference value of its own column (one parameter kind: a rotation
component, a translation component, the focal length, k1, k2; a point coordinate) over all rows.  It is the
element-wise measure for the mixed mode: FP32 Jacobians leave every element with an absolute error of the
size of its parameter kind's rounding, so an element whose own step is tiny (a point that barely moves) has
a large error relative to itself; a wrong camera or point still stands out against its column's scale."""
import numpy as np


def _ratio(d, scale):
    out = np.zeros_like(d)
    pos = scale > 0
    out[pos] = d[pos] / scale[pos]
    out[~pos & (d > 0)] = np.inf
    return float(out.max()) if out.size else 0.0


def rows(a, b, width, floor=0.0):
    """max over rows r of max_j |a_rj - b_rj| / max_j |b_rj|, rows of `width` values."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, width)
    b = np.asarray(b, dtype=np.float64).reshape(-1, width)
    assert a.shape == b.shape, (a.shape, b.shape)
    scale = np.abs(b).max(axis=1)
    if floor > 0 and b.size:
        scale = np.maximum(scale, floor * np.abs(b).max())
    return _ratio(np.abs(a - b).max(axis=1), scale)


def blocks(S, S_ref, bs=9, floor=0.0):
    """max over bs x bs blocks (I, J) of max |S_IJ - S_ref,IJ| / max |S_ref,IJ|."""
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    assert S.shape == S_ref.shape and S.shape[0] % bs == 0, (S.shape, S_ref.shape)
    nb = S.shape[0] // bs
    A = S.reshape(nb, bs, nb, bs)
    B = S_ref.reshape(nb, bs, nb, bs)
    scale = np.abs(B).max(axis=(1, 3))
    if floor > 0 and B.size:
        scale = np.maximum(scale, floor * np.abs(B).max())
    return _ratio(np.abs(A - B).max(axis=(1, 3)), scale)


def cols(a, b, width):
    """max over elements (r, j) of |a_rj - b_rj| / max_r' |b_r'j|, rows of `width` values."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, width)
    b = np.asarray(b, dtype=np.float64).reshape(-1, width)
    assert a.shape == b.shape, (a.shape, b.shape)
    scale = np.broadcast_to(np.abs(b).max(axis=0), b.shape)
    return _ratio(np.abs(a - b), scale)
