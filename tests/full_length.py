"""Comparison of a GPU state after a configuration's full step count with the
oracle's state stored by tests/golden/make_full_length.py (sampled cells,
field maxima, per-plane sums and maxima; see that script)."""
import os
import sys

import numpy as np

from parity import TOL

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if GOLDEN not in sys.path:
    sys.path.insert(0, GOLDEN)

import make_full_length as MFL  # noqa: E402  (case definitions; imports only oracle/ and workloads/)


def stored(name):
    path = os.path.join(GOLDEN, "full_length_%s.npz" % name)
    if not os.path.exists(path):
        raise FileNotFoundError("%s is missing: run tests/golden/make_full_length.py %s" % (path, name))
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def check_against_stored(u, t, steps, name, tol=TOL):
    """Assert that state u (fields, nz, ny, nx) at (t, steps) matches the
    stored oracle state of case `name`:
      * every sampled cell, per field: |u - ref| <= tol * max|ref_f| (the
        normwise per-field measure of the element-wise parity tests);
      * max |u_f| over the grid within tol * max|ref_f|;
      * on every plane normal to each axis, the sum of u_f within
        tol * max|ref_f| * (cells in the plane) and the maximum of |u_f|
        within tol * max|ref_f|.
    Returns the per-field sampled-cell errors."""
    z = stored(name)
    nf = u.shape[0]
    assert tuple(int(k) for k in z["n"]) == (u.shape[3], u.shape[2], u.shape[1]), (z["n"], u.shape)
    assert steps == int(z["steps"]), (steps, int(z["steps"]))
    assert abs(t - float(z["t"])) <= 1e-13 * max(1.0, abs(float(z["t"]))), (t, float(z["t"]))
    fmax = z["fmax"]
    assert np.all(fmax > 0)
    flat = u.reshape(nf, -1)
    err = np.abs(flat[:, z["idx"]] - z["val"]).max(axis=1) / fmax
    assert np.all(err <= tol), ("sampled cells", err)
    a = np.abs(u)
    gmax = a.reshape(nf, -1).max(axis=1)
    assert np.all(np.abs(gmax - fmax) <= tol * fmax), ("field maxima", gmax, fmax)
    for ax, axes in (("x", (1, 2)), ("y", (1, 3)), ("z", (2, 3))):
        ps, pm = u.sum(axis=axes), a.max(axis=axes)
        per_plane = u[0].size // ps.shape[1]
        ds = np.abs(ps - z["psum_" + ax]).max(axis=1)
        dm = np.abs(pm - z["pmax_" + ax]).max(axis=1)
        assert np.all(ds <= tol * fmax * per_plane), ("plane sums", ax, ds / (fmax * per_plane))
        assert np.all(dm <= tol * fmax), ("plane maxima", ax, dm / fmax)
    return err
