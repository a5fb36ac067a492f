"""Host-side parts of the tensor-based model path: the library's spectral
radius (Gelfand's formula, used by the model's renormalisation) against the
library eigenvalue routine and closed forms, and the argument checks of
cf_tm_spectral_radius.  No device use."""
import math

import numpy as np
import pytest

from oracle import tensor_model as tm


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


@pytest.mark.parametrize("dim", [1, 2, 3, 4, 7, 16])
def test_spectral_radius_matches_eigenvalues(dim):
    cf = _cf()
    rng = np.random.default_rng(dim)
    A = rng.uniform(0.05, 1.0, (dim, dim))
    assert cf.cf_tm_spectral_radius(A) == pytest.approx(tm.spectral_radius(A), rel=1e-11)


def test_spectral_radius_closed_forms():
    cf = _cf()
    assert cf.cf_tm_spectral_radius(np.diag([0.3, 4.0, 1.5])) == pytest.approx(4.0, rel=1e-12)
    assert cf.cf_tm_spectral_radius([[0.0, 1.0], [0.0, 0.0]]) == 0.0  # nilpotent
    assert cf.cf_tm_spectral_radius([[0.0, 2.0], [-2.0, 0.0]]) == pytest.approx(2.0, rel=1e-12)  # +-2i
    a, b, c, d = 1.0, 2.0, 3.0, 4.0
    lam = (a + d) / 2 + math.sqrt(((a - d) / 2) ** 2 + b * c)
    assert cf.cf_tm_spectral_radius([[a, b], [c, d]]) == pytest.approx(lam, rel=1e-12)


def test_spectral_radius_argument_checks():
    cf = _cf()
    with pytest.raises(cf.CFError) as e:
        cf.cf_tm_spectral_radius(np.array([[np.nan]]))
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError):
        cf.cf_tm_spectral_radius(np.zeros((65, 65)))
