"""The seeded input generator's Jeans dispersions satisfy the spherical Jeans equation
d(rho sigma_r^2)/dr + 2 beta rho sigma_r^2 / r = -rho G M(r) / r^2 (G = 1), checked by
finite differences, for the isotropic case (also against Hernquist 1990, eq. 10) and
for constant anisotropy."""
import numpy as np
import pytest

from paper_1202_2355_gb300 import synth


@pytest.mark.parametrize("beta", [0.0, 5.0 / 9.0, -0.5])
def test_jeans_equation_holds(beta):
    tab = synth.jeans_sigma2_table(synth.hernquist_density, synth.hernquist_mass, beta=beta)
    r = np.exp(np.linspace(np.log(0.02), np.log(20.0), 40))
    h = 0.005  # a few table segments: the table is linear in ln r between its points
    f = lambda x: synth.hernquist_density(x) * synth.sigma2_from_table(tab, x)  # noqa: E731
    lhs = (f(r * (1 + h)) - f(r * (1 - h))) / (2 * h * r) + 2 * beta * f(r) / r
    rhs = -synth.hernquist_density(r) * synth.hernquist_mass(r) / r ** 2
    assert np.allclose(lhs, rhs, rtol=1e-3)
    if beta == 0.0:
        assert np.allclose(synth.sigma2_from_table(tab, r), synth.hernquist_sigma2_iso(r), rtol=1e-4)
