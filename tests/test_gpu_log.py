"""The FP64 path's table-driven logarithm (smc_log_fp64) against a
higher-precision reference (the platform's long-double log: 64-bit mantissa
on x86, 113-bit on aarch64).  The reduction r = m G_j - 1 is exact and the
leading sum is split exactly, so the error is the final rounding (half an
ulp) plus the polynomial's truncation and the small terms' roundings
(< 2^-6 ulp): at most 0.52 ulp on the uniforms the SSA draws, on values
near 1 (where ln(1/G_j) and ln(1 + r) cancel) and on general positive
doubles, and correctly rounded on all but a few in 10^4 of them."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_log_table_accuracy():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip('no extended-precision long double on this platform')
    import paper_0912_2551_gb300 as smc
    from paper_0912_2551_gb300 import _native as N
    rng = np.random.default_rng(0)
    v = rng.integers(0, 2 ** 52, size=400000, dtype=np.uint64)
    u_ssa = (2 * v.astype(np.float64) + 1) * 2.0 ** -53          # the FP64 path's uniforms
    edges = np.array([2.0 ** -53, 1 - 2.0 ** -53, 0.5, 0.75, np.nextafter(0.75, 0), np.nextafter(0.75, 1),
                      1.0, np.nextafter(1.0, 0), 1.5, np.nextafter(1.5, 0), 2.0 / 3, 0.999, 1e-300, 1e300,
                      3.0, 1234.5678, 0.1])
    grid = 0.75 + (np.arange(193) + 0.4999) / 256                 # near table switch points
    gen = np.exp(rng.uniform(-700, 700, size=100000))
    near1 = np.concatenate([1 - (2 * rng.integers(0, 2 ** 52, size=50000, dtype=np.uint64) + 1) * 2.0 ** -59,
                            1 + (2 * rng.integers(0, 2 ** 52, size=50000, dtype=np.uint64) + 1) * 2.0 ** -59])
    u = np.concatenate([u_ssa, edges, grid, gen, near1])
    with smc.Context(0) as ctx:
        ut = torch.tensor(u, dtype=torch.float64, device='cuda')
        out = torch.empty_like(ut)
        torch.cuda.synchronize()
        rc = N.smc_log_fp64(ctx.h, ctypes.c_void_p(ut.data_ptr()), len(u), ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    ref = np.log(u.astype(np.longdouble))
    ulp = np.spacing(np.abs(ref.astype(np.float64)))
    ulp[ref == 0] = np.spacing(0.0)
    err = np.abs(got.astype(np.longdouble) - ref) / ulp.astype(np.longdouble)
    err = err.astype(np.float64)
    assert err.max() <= 0.52, (err.max(), u[err.argmax()])
    assert (err <= 0.5).mean() > 0.9995, (err <= 0.5).mean()
