"""Helpers shared by the GPU parity tests: oracle ↔ library layout conversion and tolerances."""
import numpy as np

# FP64 parity bar: iterates, gains and costs within 1e-8 relative (norm-wise per array).
RTOL64 = 1e-8

# Arrays whose exact value is zero (e.g. gains when no robust constraint is active) carry only
# rounding residue on both sides; differences below this absolute floor are not compared.
ATOL_ZERO = 1e-14


def ragged_from_dense(lin, dense):
    """Oracle (n_g, T+1, nx) row array → library ragged layout (state rows: blocks 0..t;
    control rows: block k)."""
    out = []
    for j in range(dense.shape[0]):
        t = int(lin.row_t[j])
        if j < lin.n_state:
            out.append(dense[j, :t + 1, :].reshape(-1))
        else:
            out.append(dense[j, t, :].reshape(-1))
    return np.concatenate(out) if out else np.zeros(0)


def bvec_ragged(lin):
    """Oracle b_{j,k} (state rows) → library layout: blocks 0..t, block t zero."""
    out = []
    nu = lin.bvec.shape[2]
    for j in range(lin.n_state):
        t = int(lin.row_t[j])
        blk = np.zeros((t + 1, nu))
        blk[:t] = lin.bvec[j, :t]
        out.append(blk.reshape(-1))
    return np.concatenate(out) if out else np.zeros(0)


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


# Element-wise check beside the norm-wise one: an error confined to a few entries (a short row) can
# hide under the 2-norm of a long array, which may exceed its largest entry by √n.  The max-norm
# relative error max_i |g_i - r_i| / max_i |r_i| bounds every entry's error by the same 1e-8 of the
# array's scale.  (Relative to each entry's own magnitude the bar is not meaningful: the two sides
# differ by summation order in sums whose terms have the array's scale, so the absolute rounding
# residue is about uniform over the entries.)
def max_elem_relerr(gpu, ref):
    a = np.asarray(gpu, dtype=np.float64).reshape(-1)
    b = np.asarray(ref, dtype=np.float64).reshape(-1)
    if b.size == 0:
        return 0.0
    m = np.abs(b).max()
    d = np.abs(a - b).max()
    return float(d / m) if m > 0 else float(d)


def assert_close(gpu, ref, rtol, what, atol=ATOL_ZERO, elementwise=True):
    e = relerr(gpu, ref)
    nb = np.linalg.norm(np.asarray(ref).reshape(-1))
    diff = np.linalg.norm(np.asarray(gpu, dtype=np.float64).reshape(-1) - np.asarray(ref, dtype=np.float64).reshape(-1))
    assert e <= rtol or diff <= atol, f"{what}: relative error {e:.3e} > {rtol:.1e} (|ref| = {nb:.3e})"
    if elementwise and diff > atol:
        em = max_elem_relerr(gpu, ref)
        assert em <= rtol, f"{what}: element-wise relative error {em:.3e} > {rtol:.1e}"
