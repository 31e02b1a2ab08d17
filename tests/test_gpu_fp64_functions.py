"""Accuracy of the FP64 far field's own pair functions (through the C ABI), against numpy.

The plain FP64 path takes 1/r from the MUFU rsqrt seed refined by one Newton step and
e^{-kappa r} from a 256-entry table of 2^(j/256) and a degree-4 polynomial (Tang's table-driven
method), instead of the CUDA library's sqrt, division and exp. numpy's float64 sqrt and division
are correctly rounded and its exp is within one unit in the last place, so the references below
are good to about 1 ulp. Bounds: 1/sqrt within 5 ulp; exp(-x) within 5 ulp plus the rounding of
the scaled argument, x * 2^-53 relative (the same argument rounding any exp(-kappa r) has when
kappa r is formed in double precision).
"""
import numpy as np
import pytest

from paper_1301_5914_gb300 import hobi

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def test_rsqrt_within_5_ulp():
    rng = np.random.default_rng(11)
    x = np.concatenate([10.0 ** rng.uniform(-12, 12, 400000), 4.0 ** np.arange(-20, 20),
                        1.0 + rng.uniform(0, 1, 100000), np.nextafter(1.0, 0.0) * np.ones(3)])
    rs, _ = hobi.fp64_pair_functions(x)
    ref = 1.0 / np.sqrt(x)
    err = np.abs(rs - ref) / ref
    assert np.all(np.isfinite(rs))
    assert err.max() <= 5 * ULP, err.max() / ULP
    # powers of four have exact reciprocal square roots
    p = 4.0 ** np.arange(-20, 20)
    rp, _ = hobi.fp64_pair_functions(p)
    assert np.max(np.abs(rp * np.sqrt(p) - 1.0)) <= 2 * ULP


def test_exp_within_5_ulp_plus_argument_rounding():
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(0, 50, 400000), rng.uniform(0, 700, 100000), 10.0 ** rng.uniform(-12, -1, 100000),
                        np.arange(0, 256) / 256.0 * np.log(2.0), np.array([0.0, 1.0, 2.0, 700.0])])
    _, ex = hobi.fp64_pair_functions(x)
    ref = np.exp(-x)
    err = np.abs(ex - ref) / ref
    bound = 5 * ULP + x * 2.0 ** -53
    assert np.all(err <= bound), float(np.max(err / bound))
    assert ex[x == 0.0][0] == 1.0


def test_exp_far_arguments_stay_finite_and_tiny():
    # padding nodes and distant pairs: the argument is clamped so the result stays a tiny normal double
    x = np.array([745.0, 1e3, 1e4, 1e6, 1e9, 1e12])
    rs, ex = hobi.fp64_pair_functions(x)
    assert np.all(np.isfinite(ex)) and np.all(ex > 0.0) and np.all(ex <= 1e-300)
    assert np.all(ex * 1e300 < 1.0)


def test_argument_errors():
    with pytest.raises(hobi.HobiError):
        hobi.fp64_pair_functions(np.array([-1.0]))
    with pytest.raises(hobi.HobiError):
        hobi.fp64_pair_functions(np.array([np.nan]))
    with pytest.raises(hobi.HobiError):
        hobi.fp64_pair_functions(np.array([1e13]))
    rs, ex = hobi.fp64_pair_functions(np.zeros(0))
    assert rs.size == 0 and ex.size == 0
