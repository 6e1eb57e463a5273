"""Direct accuracy test of the library's float-float exponential (the Gaussian delta weights
of the FP64-grade rate epilogue, Eq. X^e-ph with reading [A10]) through the C ABI.

The kernel takes its input as a float-float pair, so the test draws inputs that are exact
float-float values (hi + lo with lo below half an ulp of hi) and compares with the FP64
exponential of that exact value.  Bound: the argument reduction y = k ln 2 + r subtracts k ln 2
in three parts (two exact FP32 products and a rounded third), so r carries ~2^-49 absolute
error; the 13-term float-float Horner steps add a few 2^-48 of e^r: 2^-45 relative overall,
whatever |y|."""
import numpy as np
import pytest

from paper_2109_08547_gb300 import binding as B

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -45


def _exact_ff_inputs(n, rng):
    hi = rng.uniform(-60.0, 0.0, n).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    y = hi.astype(np.float64) + lo.astype(np.float64)
    # the grid ends and a few exact values
    extra = np.array([0.0, -1e-30, -0.5 * np.log(2.0), -np.log(2.0), -1.0, -8.0, -32.0, -59.999, -60.0])
    extra = extra.astype(np.float32).astype(np.float64)
    return np.concatenate([y, extra])


def test_exp_ff_relative_error_over_its_range():
    import torch
    rng = np.random.default_rng(2109)
    y = _exact_ff_inputs(1 << 20, rng)
    yd = torch.from_numpy(y).cuda()
    out = torch.empty_like(yd)
    assert B.selftest_exp_ff(yd.data_ptr(), out.data_ptr(), len(y)) == B.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.exp(y)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= BOUND, (rel.max(), y[np.argmax(rel)])
    # the half of the range the 8-sigma Gaussian uses (-32 <= y <= 0) keeps the same bound
    assert np.all(got[y == 0.0] == 1.0)


def test_exp_ff_argument_errors():
    assert B.selftest_exp_ff(0, 0, -1) == B.EINVAL
    assert B.selftest_exp_ff(0, 0, 4) == B.EINVAL
    assert B.selftest_exp_ff(0, 0, 0) == B.OK
