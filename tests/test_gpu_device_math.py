"""The binary32 square roots of the kernels (gamma = sqrt(1 + p^2), |p|, 1/gamma): the
hardware reciprocal-square-root estimate refined by one Newton step, checked through
sfq_check_sqrt against correctly rounded results over the normal binary32 range.

The reference is the binary64 square root of the binary32 input rounded to binary32:
rounding a correctly rounded 53-bit square root to 24 bits gives the correctly rounded
24-bit one (53 >= 2 * 24 + 2), so it is the IEEE result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(n=1 << 20, seed=5):
    rng = np.random.default_rng(seed)
    bits = (rng.integers(1, 254, n, dtype=np.uint32) << 23) | rng.integers(0, 1 << 23, n, dtype=np.uint32)
    x = bits.view(np.float32)
    special = np.array([1.0, 2.0, 4.0, 0.25, np.nextafter(np.float32(1), np.float32(2)),
                        np.nextafter(np.float32(1), np.float32(0)), 1.17549435e-38, 3.4e38, 1e-20, 1e20,
                        1.0 + 4e6 ** 2], np.float32)
    # gamma^2 = 1 + p^2 of the configs' momenta (|p| from 1e-3 to 1e7)
    p = np.exp(rng.uniform(np.log(1e-3), np.log(1e7), 1 << 16)).astype(np.float32)
    g2 = (np.float32(1) + p * p).astype(np.float32)
    return np.concatenate([x, special, g2])


def _ulps(a, b):
    return np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64))


def test_sqrt_and_rsqrt_within_one_ulp():
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=0.8e-6, dt=1e-17, precision="fp32", seed=1)
    x = _inputs()
    s, r = ctx.check_sqrt(torch.as_tensor(x, device=ctx.device))
    s, r = s.cpu().numpy(), r.cpu().numpy()
    want_s = np.sqrt(x.astype(np.float64)).astype(np.float32)
    want_r = (1.0 / np.sqrt(x.astype(np.float64))).astype(np.float32)
    us, ur = _ulps(s, want_s), _ulps(r, want_r)
    assert us.max() <= 1, (us.max(), x[us.argmax()], s[us.argmax()], want_s[us.argmax()])
    assert ur.max() <= 1, (ur.max(), x[ur.argmax()], r[ur.argmax()], want_r[ur.argmax()])
    # most results are the correctly rounded ones
    assert (us == 0).mean() > 0.9 and (ur == 0).mean() > 0.8, ((us == 0).mean(), (ur == 0).mean())
    ctx.close()


def test_sqrt_of_non_positive_is_zero():
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=0.8e-6, dt=1e-17, precision="fp32", seed=1)
    x = np.array([0.0, -0.0, -1.0, -3e38, np.nan], np.float32)
    s, _ = ctx.check_sqrt(torch.as_tensor(x, device=ctx.device))
    assert np.array_equal(s.cpu().numpy(), np.zeros(5, np.float32))
    assert ctx.check_sqrt(torch.empty(0, device=ctx.device))[0].numel() == 0
    ctx.close()
