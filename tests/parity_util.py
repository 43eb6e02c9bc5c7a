"""Population parity checks shared by the GPU tests (not collected by pytest).

Two measures of a GPU population field f_d against the FP64 oracle's f_o,
both [19][z][y][x], unshifted:

* the relative L2 error ||f_d - f_o|| / ||f_o|| (the metric the 1e-6 FP32
  bound is stated in).  The lattice weights dominate ||f_o|| (sqrt(sum w_i^2)
  per cell), so this alone would let one population of one cell be off by
  about 1e-6 * ||f_o||;
* the largest single error, max |f_d - f_o|, against the largest offset from
  the weights, max |f_o - w|: one element wrong anywhere, a boundary row
  included, fails it.

ELEM_TOL, the bound of the second measure for FP32 compute with FP32 storage
over 100 steps: each step stores f - w rounded to FP32 (half an ulp, 6e-8 of
the value) after some 30 FP32 operations on quantities of the size of f - w
(the approximate division and square root add about 2 ulp), so a step adds
at most a few 1e-7 of max |f - w| per element.  BGK relaxation with
tau_total near 1/2 damps these errors barely (the factor 1 - 1/tau is near
-1), so over 100 steps they add up to at most 100 times that, a few 1e-5 in
the worst case, and about 10 times that for a random walk.  1e-4 stays above
the worst case and is four orders of magnitude tighter than what the relative
L2 bound allows for one element.
"""
import numpy as np

ELEM_TOL = 1e-4
W_LATTICE = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def population_errors(fd, fo):
    """(relative L2, max |fd - fo| / max |fo - w|, location (q, z, y, x) of the
    largest error, per-region maxima / max |fo - w|), one direction plane at
    a time to bound the memory."""
    num = den = 0.0
    worst, where, scale = -1.0, None, 0.0
    regions = {"y=0": 0.0, "y=top": 0.0, "x=0": 0.0, "x=last": 0.0, "z=0": 0.0}
    for q in range(fd.shape[0]):
        d = np.abs(fd[q] - fo[q])
        num += float(np.sum(d * d))
        den += float(np.sum(fo[q] * fo[q]))
        scale = max(scale, float(np.abs(fo[q] - W_LATTICE[q]).max()))
        k = int(np.argmax(d))
        if d.flat[k] > worst:
            worst, where = float(d.flat[k]), (q,) + tuple(int(i) for i in np.unravel_index(k, d.shape))
        regions["y=0"] = max(regions["y=0"], float(d[:, 0, :].max()))
        regions["y=top"] = max(regions["y=top"], float(d[:, -1, :].max()))
        regions["x=0"] = max(regions["x=0"], float(d[:, :, 0].max()))
        regions["x=last"] = max(regions["x=last"], float(d[:, :, -1].max()))
        regions["z=0"] = max(regions["z=0"], float(d[0].max()))
    scale = max(scale, 1e-300)
    return (np.sqrt(num / den), worst / scale, where,
            {k: v / scale for k, v in regions.items()})


def assert_population_parity(fd, fo, l2_tol=1e-6, elem_tol=ELEM_TOL, label=""):
    """Both measures within their bounds; the message names the worst element."""
    l2, elem, where, regions = population_errors(fd, fo)
    msg = (f"{label}: rel L2 {l2:.2e} (bound {l2_tol:.0e}), max element error {elem:.2e} of "
           f"max|f-w| (bound {elem_tol:.0e}) at (q,z,y,x)={where}; by boundary row "
           + " ".join(f"{k}:{v:.1e}" for k, v in regions.items()))
    print(msg)
    assert l2 <= l2_tol, msg
    assert elem <= elem_tol, msg
    return l2, elem
