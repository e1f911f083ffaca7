"""Shared test helpers: tolerance rule and comparison of the CUDA path's
outputs with the FP64 oracle."""
import numpy as np

# SNR agreement bar for the FP32 path: |delta| <= 1e-5 * max(1, |SNR_oracle|)
# (relative 1e-5, absolute 1e-5 in sigma units below |SNR| = 1).
SNR_TOL = 1e-5
# argmax must agree wherever the two best filters differ by more than this
ARGMAX_GAP = 1e-3


def snr_close(got, want, tol=SNR_TOL):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
    return err, bool(np.all(err <= tol))


def top2_gap(snr, valid):
    """Gap between best and second-best valid SNR per pixel (inf if < 2 valid)."""
    s = np.where(valid, snr, -np.inf)
    part = np.sort(s, axis=0)
    top1, top2 = part[-1], part[-2] if s.shape[0] > 1 else np.full(s.shape[1:], -np.inf)
    with np.errstate(invalid="ignore"):
        gap = top1 - top2
    return np.where(np.isfinite(top2), gap, np.inf)


def check_search(got_max, got_arg, got_all, N, D, oracle, tol=SNR_TOL, label=""):
    snr, valid, smax, amax = oracle.snr_and_best(N, D)
    err, ok = snr_close(got_max, smax, tol)
    assert ok, "%s snr_max max rel err %.3g at %s" % (label, err.max(), np.unravel_index(err.argmax(), err.shape))
    gap = top2_gap(snr, valid)
    decided = gap > ARGMAX_GAP
    none = amax < 0
    assert np.array_equal(got_arg[none], amax[none]), label + " argmax -1 pixels differ"
    bad = decided & (got_arg != amax)
    assert not bad.any(), "%s argmax differs at %d decided pixels, e.g. %s" % (
        label, bad.sum(), np.argwhere(bad)[:3].tolist())
    # where the decision is close, the chosen filter must still be (near) best
    kk = np.where(got_arg >= 0, got_arg, 0)
    chosen = np.take_along_axis(snr, kk[None], 0)[0]
    close = (~decided) & (~none)
    assert np.all(np.abs(chosen[close] - smax[close]) <= ARGMAX_GAP + tol * np.maximum(1, np.abs(smax[close])))
    if got_all is not None:
        err, ok = snr_close(got_all, snr, tol)
        assert ok, "%s snr_all max rel err %.3g at %s" % (label, err.max(), np.unravel_index(err.argmax(), err.shape))
    return err
