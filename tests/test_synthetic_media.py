"""The separable lattice-well generators equal the direct sum over wells (same seed,
same depths): they only reorder the arithmetic of synthetic_media's plain form."""
import numpy as np
import pytest

import synthetic_media as sm


@pytest.mark.parametrize("n,ell", [(16, 2.0), (32, 4.0), (48, 8.0)])
def test_wells_2d_separable(n, ell):
    a = sm.lattice_wells_potential(2, n, ell, 1234)
    b = sm.lattice_wells_potential_2d(n, ell, 1234)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("n,ell", [(16, 2.0), (24, 4.0), (32, 4.0)])
def test_wells_3d_separable(n, ell):
    a = sm.lattice_wells_potential(3, n, ell, 1000)
    b = sm.lattice_wells_potential_3d(n, ell, 1000)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
