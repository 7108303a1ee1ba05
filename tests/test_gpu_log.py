"""The FP64 path's logarithm (smc_log_fp64: table-driven, evaluated on the
integer pipes) against a higher-precision reference (the platform's
long-double log: 64-bit mantissa on x86, 113-bit on aarch64).  The
reduction r = m G_j - 1 is exact and the sum is formed in 128-bit fixed
point, so the error is the final rounding (half an ulp) plus under 2^-9 ulp:
at most 0.502 ulp on the uniforms the SSA draws, on values near 1 (where
ln(1/G_j) and ln(1 + r) cancel) and on general positive doubles, and
correctly rounded on all but about one in 10^5 of them.  The division of the
same step (smc_div_fp64) must give the IEEE-754 quotient bit for bit."""
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
    assert err.max() <= 0.502, (err.max(), u[err.argmax()])
    assert (err <= 0.5).mean() > 0.9999, (err <= 0.5).mean()



def test_division_is_ieee():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    from paper_0912_2551_gb300 import _native as N
    rng = np.random.default_rng(1)
    n = 1 << 21
    bits = rng.integers(0, 2 ** 63, size=(2, n), dtype=np.uint64)
    anyclass = bits.view(np.float64)                                  # every class, both signs
    frac = rng.integers(0, 2 ** 52, size=(2, n), dtype=np.uint64)
    expo = rng.integers(1023 - 40, 1023 + 40, size=(2, n), dtype=np.uint64)
    moderate = ((expo << np.uint64(52)) | frac).view(np.float64)      # positive normals
    q = moderate[0] * moderate[1]                                      # exact-ish quotients and neighbours
    near = (q.view(np.uint64) + rng.integers(-2, 3, size=n).astype(np.uint64)).view(np.float64)
    taus = np.stack([-np.log((2 * rng.integers(0, 2 ** 52, size=n, dtype=np.uint64).astype(np.float64) + 1)
                             * 2.0 ** -53), np.exp(rng.uniform(-5, 12, size=n))])  # -ln u / a_0 of the SSA
    edges = np.array([[1.0, 3.0], [1.0, 1.0], [3.0, 2.0], [1e308, 1e-10], [1e-300, 1e10], [2.0 ** -1022, 2.0],
                      [4.0, 2.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 3.0], [np.inf, 2.0], [np.nan, 1.0],
                      [1.9999999999999998, 1.0000000000000002], [5e-324, 1.0]]).T
    num = np.concatenate([anyclass[0], moderate[0], near, taus[0], edges[0]])
    den = np.concatenate([anyclass[1], moderate[1], moderate[1], taus[1], edges[1]])
    with smc.Context(0) as ctx:
        a = torch.tensor(num, dtype=torch.float64, device='cuda')
        b = torch.tensor(den, dtype=torch.float64, device='cuda')
        out = torch.empty_like(a)
        torch.cuda.synchronize()
        rc = N.smc_div_fp64(ctx.h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(),
                            ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0
        want = (a / b).cpu().numpy()
        got = out.cpu().numpy()
    same = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
    assert same.all(), (num[~same][:4], den[~same][:4], got[~same][:4], want[~same][:4])
