"""Bars for comparing a GPU Krylov solve with the oracle's run of the same method.

The two runs are different, equally valid roundings of the method: the GPU reduces every inner
product in a fixed tree order (leaves of 16, pairwise tree) and the oracle sums left to right
(Algorithm 3's plain sum), so a scalar such as rho = <r~, r> may differ in its last DD bits.
What the stated tolerances ask, and what these helpers assert:

  * the recursive residual norms ||r_k|| (leading components) agree within 1e-10 relative for
    k = 0 .. 20 ("band"), while ||r_k|| / ||r_0|| is above the floor stated below;
  * the iteration counts agree within 5 % (at least 1);
  * both runs end with the same status, and a converged run's true residual ||b - A x|| is
    within 10x the target (the replacement rule's acceptance level);
  * on well-conditioned systems the final error against x* meets the format's bound.

Floors of the band (measured properties of the method, not of either implementation):
  * binary32 / bfloat16 factors: the right-hand side of M^-1 is rounded to binary32.  Once
    ||r_k|| / ||r_0|| is near 1e-20, the DD-level difference between the two runs' r decides
    some of those roundings differently, and the runs separate at the binary32 level (measured
    at 33 x 33: first visible between 6e-20 and 3e-24).  Band floor 1e-15: there the expected
    number of flipped roundings per application, n * 2^-53 / (2^-24 * 1e-15), is below 1e-3 for
    n <= 4e6.
  * D vectors (w = 1): the residual norm itself carries a relative error ~ u / (||r_k|| / ||r_0||),
    u = 2^-53; band floor 1e-4.
  * indefinite systems (the shifted-Laplacian Helmholtz matrices): the iteration amplifies a
    one-rounding difference in an inner product by 20-50x per iteration (measured on a 23 x 23
    grid: 1e-31 in the iterate after one iteration, 2e-14 after fifteen), so the band holds for
    the first 12 iterations only and the iteration counts of two valid runs differ by up to 20 %.
"""
import numpy as np

BAND = 1e-10
LP_FLOOR = 1e-15


def band_floor(ilu, w):
    """Relative residual level above which the band is asserted."""
    f = 2.0 ** (-53 * w) * 1e12  # D: 1.1e-4; DD: 1.2e-20; TD, QD: below any target used here
    if ilu in ("fp32", "bf16"):
        f = max(f, LP_FLOOR)
    return f


def check_band(hist_gpu, hist_ref, floor, kmax=20):
    """||r_k|| within BAND relative for k <= kmax while ||r_k|| / ||r_0|| >= floor."""
    g = np.asarray(hist_gpu, dtype=np.float64)
    r = np.asarray(hist_ref, dtype=np.float64)
    m = min(kmax + 1, len(g), len(r))
    assert m >= 1
    checked = 0
    for k in range(m):
        if r[k] < floor * r[0] or g[k] < floor * g[0]:
            break
        assert abs(g[k] - r[k]) <= BAND * r[k], (k, g[k], r[k], abs(g[k] - r[k]) / r[k])
        checked += 1
    return checked


def check_iters(it_gpu, it_ref, frac=0.05):
    assert abs(it_gpu - it_ref) <= max(1, int(frac * it_ref)), (it_gpu, it_ref)


def check_solve(out, ref, ilu, w, tol, indefinite=False, same_status=True):
    """The stated bars for one GPU solve `out` against the oracle's `ref` (dicts with status,
    iters, hist, relres_true)."""
    if same_status:
        assert out["status"] == ref["status"], (out["status"], ref["status"])
    floor = band_floor(ilu, w)
    check_band(out["hist"], ref["hist"], floor, kmax=12 if indefinite else 20)
    if out["status"] == "OK" and ref["status"] == "OK":
        check_iters(out["iters"], ref["iters"], 0.2 if indefinite else 0.05)
    return floor


def rel_error(x, x_star, n, c, w):
    """max_i |x_i - x*_i| / max_i |x*_i| with x, x* as n*c*w components; each difference is the
    correctly rounded value difference of the two w-component numbers (mp_diff)."""
    S = np.asarray(x_star, dtype=np.float64).reshape(n, c, w)
    err = np.abs(mp_diff(x, x_star, w)).max()
    return err / np.abs(S[:, :, 0]).max()


def mp_diff(y, ref, w):
    """Value differences of multi-component numbers, entry by entry: sum_k y_k - sum_k ref_k
    correctly rounded (math.fsum over the 2w components).  Two representations of one value may
    split it differently between components (the device's TD / QD renormalisation and the
    oracle's greedy rounding do), so components are never compared one by one."""
    import math

    Y = np.asarray(y, dtype=np.float64).reshape(-1, w)
    R = np.asarray(ref, dtype=np.float64).reshape(-1, w)
    if w == 1:
        return Y[:, 0] - R[:, 0]
    both = np.concatenate([Y, -R], axis=1)
    return np.array([math.fsum(row) for row in both])
