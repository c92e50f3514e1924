"""The reciprocals behind every Cholesky pivot and Householder scalar of the
factor kernels (Sec. 2: the diagonal blocks A_ss = G_s G_s^T; Sec. 3.1: the
column-pivoted QR), checked directly rather than only through end-to-end
parity: an FP32 estimate refined by two Newton-Raphson steps must land within
one unit in the last place (ulp) of the exact 1/x and two ulp of the exact
1/sqrt(x), and agree with CUDA's own FP64 division and rsqrt to the same
bounds.  The exact values come from numpy's extended precision (80-bit on
x86, 128-bit on aarch64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    from paper_1811_11248_gb300 import build, hsolve
    build.build()
    hsolve.lib()
    assert torch.cuda.is_available()
    return hsolve


def _inputs():
    rng = np.random.default_rng(11)
    parts = [
        10.0 ** rng.uniform(-300, 300, 400_000),  # the whole positive range
        10.0 ** rng.uniform(-3, 3, 400_000),      # typical pivots
        np.ldexp(1.0, np.arange(-990, 990)),       # powers of two
        1.0 + np.ldexp(rng.integers(-2**20, 2**20, 20_000).astype(float), -52),  # next to 1
        # the edges of the FP32-seeded range and of the FP32 exponent range
        np.concatenate([e * (1.0 + np.ldexp(np.arange(-200, 200, dtype=float), -40))
                        for e in (1e-30, 1e30, 1.1754943508222875e-38, 3.4028234663852886e38)]),
    ]
    x = np.concatenate(parts)
    return x[(x > 0) & np.isfinite(x)]


def _ulp_err(y, exact):
    """|y - exact| in units of the spacing of the FP64 numbers at exact."""
    ex = exact.astype(np.float64)
    return (np.abs(y.astype(np.longdouble) - exact) / np.spacing(np.abs(ex)).astype(np.longdouble)).astype(np.float64)


def test_pivot_reciprocals_within_ulp_bounds(hs):
    x = _inputs()
    xd = torch.from_numpy(x).cuda()
    rs = torch.empty_like(xd)
    rc = torch.empty_like(xd)
    hs.hs_eval_pivot_reciprocals(xd, rs, rc)
    rs_h, rc_h = rs.cpu().numpy(), rc.cpu().numpy()
    xl = x.astype(np.longdouble)
    e_rs = _ulp_err(rs_h, 1 / np.sqrt(xl))
    e_rc = _ulp_err(rc_h, 1 / xl)
    print(f"max ulp error: 1/sqrt {e_rs.max():.3f}, 1/x {e_rc.max():.3f} over {len(x)} inputs")
    assert np.all(np.isfinite(rs_h)) and np.all(np.isfinite(rc_h))
    assert e_rc.max() <= 1.0
    assert e_rs.max() <= 2.0
    # CUDA's own FP64 operations on the same device
    cuda_rc = (1.0 / xd).cpu().numpy()
    cuda_rs = torch.rsqrt(xd).cpu().numpy()
    sp = np.spacing(np.abs(cuda_rc))
    assert np.max(np.abs(rc_h - cuda_rc) / sp) <= 1.0
    sp = np.spacing(np.abs(cuda_rs))
    assert np.max(np.abs(rs_h - cuda_rs) / sp) <= 2.0 + 1.0  # CUDA's rsqrt is itself within 1 ulp
