"""The library's fitted tables in both bases (sfq_table_pieces, host only, no GPU): every
piece converted to the Chebyshev basis is the same polynomial as its monomial form.

Checked against numpy's own evaluators (polyval / polyval2d on the monomial pieces,
chebval / chebval2d on the Chebyshev pieces) at random points of [-1, 1] (squared for the
inverse-CDF pieces): the two agree to the rounding of the coefficients, measured against
eps times the sum of the Chebyshev coefficients' magnitudes, a bound on the piece's values.
A dropped term, a transposed operand or a wrong recurrence would differ by the size of a
coefficient.  The padding of the inverse-CDF rows stays zero in both bases.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as Ch
from numpy.polynomial import polynomial as Pm

# coefficients per variable: rates (degree 8 / 10) and inverse CDFs (9 x 9 / 12 x 12)
SHAPES = {"fp32": (9, 9), "fp64": (11, 12)}
EPS = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
SLACK = {"fp32": 2.0, "fp64": 32.0}          # measured worst: 0.93 and 7.7


@pytest.fixture(scope="module")
def sfq():
    from paper_2301_07684_gb300 import build
    build.build()
    from paper_2301_07684_gb300 import sfq as S
    return S


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_chebyshev_pieces_are_the_monomial_pieces(sfq, precision, which):
    nr, ni = SHAPES[precision]
    m = sfq.table_pieces(precision, which, sfq.SFQ_EVAL_HORNER).astype(np.float64)
    c = sfq.table_pieces(precision, which, sfq.SFQ_EVAL_CLENSHAW).astype(np.float64)
    assert m.size == c.size > 0
    g = np.random.default_rng(which)
    tol = SLACK[precision] * EPS[precision]
    if which < 2:
        M, C = m.reshape(-1, nr), c.reshape(-1, nr)
        x = np.concatenate([[-1.0, 0.0, 1.0], g.uniform(-1, 1, 6)])
        for p in range(M.shape[0]):
            d = np.abs(Pm.polyval(x, M[p]) - Ch.chebval(x, C[p])).max()
            assert d <= tol * np.abs(C[p]).sum(), (p, d)
    else:
        esz = 4 if precision == "fp32" else 8
        row = (ni * esz + 15) // 16 * 16 // esz
        M, C = m.reshape(-1, ni, row), c.reshape(-1, ni, row)
        assert not M[:, :, ni:].any() and not C[:, :, ni:].any()
        x = np.concatenate([[-1.0, 1.0, 0.0], g.uniform(-1, 1, 4)])
        y = np.concatenate([[1.0, -1.0, 0.0], g.uniform(-1, 1, 4)])
        for p in range(M.shape[0]):
            d = np.abs(Pm.polyval2d(x, y, M[p, :, :ni]) - Ch.chebval2d(x, y, C[p, :, :ni])).max()
            assert d <= tol * np.abs(C[p, :, :ni]).sum(), (p, d)


def test_table_query_and_errors(sfq):
    import ctypes as C
    n = C.c_size_t(0)
    assert sfq.lib().sfq_table_pieces(sfq.SFQ_FP32, 0, 0, None, C.byref(n)) == 0 and n.value > 0
    small = (C.c_ubyte * 8)()
    n2 = C.c_size_t(8)
    assert sfq.lib().sfq_table_pieces(sfq.SFQ_FP32, 0, 0, small, C.byref(n2)) == 3          # SFQ_ERR_CAPACITY
    assert n2.value == n.value
    for bad in ((7, 0, 0), (sfq.SFQ_FP32, 4, 0), (sfq.SFQ_FP32, 0, 2)):
        assert sfq.lib().sfq_table_pieces(*bad, None, C.byref(n)) == 1                      # SFQ_ERR_ARG
    assert sfq.lib().sfq_table_pieces(sfq.SFQ_FP32, 0, 0, None, None) == 1
