"""The stored exact integer product (tests/golden, Eq. 5) through the GPU forms:
naive FP64 bit-exact, FFT-CONV in FP64 and split form exact after rounding."""
import numpy as np
import pytest

from tests.gpu_util import dev, host
from tests.test_golden import load_star_fixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def test_gpu_forms_reproduce_the_stored_product(nspt):
    A, B, C = load_star_fixture()
    A2, B2, C2 = (np.stack([X, X]) for X in (A, B, C))   # batch of 2
    np.testing.assert_array_equal(host(nspt.polymat_mul(dev(A2), dev(B2), algo="naive")), C2)
    for prec, tol in (("fp64", 1e-9), ("split", 1e-6)):
        D = host(nspt.polymat_mul(dev(A2), dev(B2), algo="fft", prec=prec))
        assert np.abs(D - C2).max() < tol, prec
        np.testing.assert_array_equal(np.round(D.real) + 1j * np.round(D.imag), C2)
