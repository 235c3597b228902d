"""Shared helpers of the GPU parity tests: load the library, compare with the oracle."""
import numpy as np
import pytest

from oracle import gustavson as og

TOL_F64 = 1e-12   # |c - c_ref| <= TOL * (|A||B|)_ij
TOL_F32 = 2e-6
WARP_ROW_OUTPUTS = 675   # row kernels: warp tables up to this many outputs (SGC_WARP_ROW_OUTPUTS), atomics above


def lib():
    """Builds (if stale) and imports the binding; skips when no CUDA device."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21253_gb300 import build
    build.build()
    from paper_2507_21253_gb300 import sgc
    return sgc


def compare(C, A, B, rows=None, tol=None, exact_f64=False):
    """C (DeviceCsr) against the oracle's A*B on all rows or on `rows`.

    Structure must match exactly; int64 values exactly; floating values within
    tol * (|A||B|)_ij (FP64 reference for FP32).  Returns the fraction of FP
    values that are bit-identical to the FP64 oracle (FP64 inputs)."""
    rp, col, val = C.to_host()
    orp, ocol, oval, omag = og.spgemm(A, B, rows=rows)
    if rows is None:
        assert np.array_equal(rp, orp), "row pointer differs"
        assert np.array_equal(col, ocol), "column ids differ"
        got = val
    else:
        segs_c, segs_v = [], []
        for s, r in enumerate(rows):
            a, b = rp[r], rp[r + 1]
            assert b - a == orp[s + 1] - orp[s], f"row {r}: count {b - a} vs {orp[s + 1] - orp[s]}"
            segs_c.append(col[a:b])
            segs_v.append(val[a:b])
        got_c = np.concatenate(segs_c) if segs_c else np.zeros(0, np.int32)
        assert np.array_equal(got_c, ocol), "column ids differ"
        got = np.concatenate(segs_v) if segs_v else val[:0]
    if val.dtype == np.int64:
        assert np.array_equal(got, oval), "int64 values differ"
        return 1.0
    if tol is None:
        tol = TOL_F32 if val.dtype == np.float32 else TOL_F64
    err = np.abs(got.astype(np.float64) - oval)
    bad = err > tol * omag
    assert not bad.any(), f"{int(bad.sum())} values beyond {tol}*(|A||B|): max rel {float((err / np.maximum(omag, 1e-300)).max())}"
    same = float(np.mean(got.astype(np.float64) == oval)) if got.size else 1.0
    if exact_f64:
        # rows computed row by row with more than WARP_ROW_OUTPUTS outputs accumulate
        # with shared-memory atomics (order not fixed); every other row is bit-identical
        counts = np.diff(orp)
        fixed = np.repeat(counts <= WARP_ROW_OUTPUTS, counts)
        eq = got.astype(np.float64) == oval
        assert eq[fixed].all(), f"only {float(eq[fixed].mean()):.6f} of FP64 values bit-identical"
    return same


def sample_rows(n, k, seed):
    rs = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rs.integers(0, n, size=min(k, n))])).astype(np.int64)
