"""Barree-Conway apparent-permeability model (Eq. AppPer, normalised as Eq.
normalizedPermeability) and its least-squares fit.

The oracle's model is pinned by its limits (Darcy plateau K* = 1 at Re -> 0, the
minimum m at Re -> infinity, the value at the transition a Re = 1) and its fit by
recovering the parameters of noiseless data it did not see fitted before.  The library's
fit (host code behind the C ABI, no GPU) must then agree with the oracle's on the same
data, noiseless and noisy.
"""
import numpy as np
import pytest

TRUE = (0.18, 0.02, 0.7, 1.6)     # m, a, E, F


def _data(n=24, noise=0.0, seed=0):
    import oracle
    re = np.logspace(-2, 3.5, n)
    k = oracle.barree_conway(re, *TRUE)
    if noise:
        k = k + noise * np.random.default_rng(seed).standard_normal(n)
    return re, k


def test_model_limits(orc):
    m, a, E, F = TRUE
    assert orc.barree_conway(1e-12, *TRUE) == pytest.approx(1.0, abs=1e-12)
    assert orc.barree_conway(1e12, *TRUE) == pytest.approx(m, abs=1e-6)
    assert orc.barree_conway(1.0 / a, *TRUE) == pytest.approx(m + (1 - m) * 2.0 ** -E, rel=1e-15)
    k = orc.barree_conway(np.logspace(-3, 5, 50), *TRUE)
    assert np.all(np.diff(k) < 0)


def test_oracle_fit_recovers_parameters(orc):
    re, k = _data()
    p, rms = orc.fit_barree_conway(re, k, init=[0.3, 0.05, 1.0, 1.0])
    assert np.allclose(p, TRUE, rtol=1e-7, atol=0)
    assert rms < 1e-12


@pytest.mark.parametrize("noise", [0.0, 2e-3])
def test_library_fit_matches_oracle(orc, noise):
    from paper_1508_02960_gb300 import capi
    capi.lib(build_if_missing=True)
    re, k = _data(noise=noise, seed=7)
    init = [0.3, 0.05, 1.0, 1.0]
    p_or, rms_or = orc.fit_barree_conway(re, k, init=init)
    p_lib, rms_lib = capi.fit_barree_conway(re, k, init=init)
    assert np.allclose(p_lib, p_or, rtol=1e-5, atol=1e-9), (p_lib, p_or)
    assert rms_lib == pytest.approx(rms_or, rel=1e-6, abs=1e-14)
    if noise == 0.0:
        assert np.allclose(p_lib, TRUE, rtol=1e-7, atol=0)
    p_def, _ = capi.fit_barree_conway(re, k)       # default starting guess
    assert np.allclose(p_def, p_or, rtol=1e-4, atol=1e-8)


def test_library_fit_rejects_bad_input():
    from paper_1508_02960_gb300 import capi
    with pytest.raises(capi.LBMError):
        capi.fit_barree_conway([1.0, 2.0, 3.0], [1.0, 0.9, 0.8])
    with pytest.raises(capi.LBMError):
        capi.fit_barree_conway([1.0, -2.0, 3.0, 4.0], [1.0, 0.9, 0.8, 0.7])
