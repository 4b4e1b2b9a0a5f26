"""ugkwp_get_field_noalloc (fixed device scratch, no allocation) against ugkwp_get_field.

Collected last (file name) so that it also runs after every other GPU test has used the device; it passes
on its own as well. Tolerance: both calls run the same conversion kernel on the same state, so the values
agree to the last bit; the bar is rtol 1e-14."""
import numpy as np
import pytest

from paper_2607_09552_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_field_equals_field_on_two_calls_in_a_row(cuda_lib, prec):
    case = wl.case_cylinder(19, 26, 0.01, 6.0, Kn=0.05, Ma=5.0, n_ref=20)
    s = cuda_lib.Solver(case, precision=prec)
    s.step(4)
    W, Wp = s.field()
    for _ in range(2):
        W2, Wp2 = s.field_noalloc()
        np.testing.assert_allclose(W2, W, rtol=1e-14, atol=0)
        np.testing.assert_allclose(Wp2, Wp, rtol=1e-14, atol=1e-300)
    assert np.any(Wp != 0)
    # and again after the state moved on
    s.step(2)
    W, Wp = s.field()
    W2, Wp2 = s.field_noalloc()
    np.testing.assert_allclose(W2, W, rtol=1e-14, atol=0)
    np.testing.assert_allclose(Wp2, Wp, rtol=1e-14, atol=1e-300)
    W3, none = s.field_noalloc(with_wp=False)
    assert none is None
    np.testing.assert_allclose(W3, W, rtol=1e-14, atol=0)


def test_noalloc_rejects_meshes_beyond_its_scratch(cuda_lib):
    case = wl.case_cylinder(320, 320, 1e-3, 15.0, Kn=0.1, Ma=5.0, n_ref=4)   # 102400 cells > 98304
    s = cuda_lib.Solver(case, precision=0, wave_only=True)
    with pytest.raises(cuda_lib.UgkwpError) as e:
        s.field_noalloc()
    assert e.value.status == 1 and "98304" in str(e.value)
    W, _ = s.field()   # the allocating entry point still serves it
    # a W-only call uses no scratch, so it serves any mesh
    W2, none = s.field_noalloc(with_wp=False)
    assert none is None
    np.testing.assert_array_equal(W2, W)
