"""Pin of the upwinding direction of the shift advection (Sec. 3: the advection terms
beta^k d_k use upwind-biased stencils).  Upwind- and downwind-biased 4th-order stencils
agree to O(h^4) on smooth data, so convergence tests cannot tell them apart; at the
grid's highest frequency they differ in sign.  An upwinded beta^z d_z damps the mode
(-1)^i2 for either sign of beta^z, while a downwinded one would amplify it.

State: flat conformal data (h = a = 0, W = alpha = 1, Lambdabar = B = 0), a constant
Cartesian shift beta^z = +-0.5 on a SinhCylindrical grid (its z frame vector is the
Cartesian one), K = eps (-1)^i2, no dissipation.  Then d_t K = beta^z e_z K + K^2/3
exactly (every other term of Eq. K_RHS vanishes), so d_t K - K^2/3 is the advection."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_00097_gb300 import workloads as W


@pytest.mark.parametrize("bz", [0.5, -0.5])
@pytest.mark.parametrize("ng", [3, 5])
def test_upwinded_advection_damps_the_highest_frequency(bz, ng):
    spec = W.sinh_cylindrical((8, 4, 24), rho_max=6.0, z_max=6.0, ko_sigma=0.0)
    spec["NG"] = ng
    o = Oracle(spec)
    T = o.T
    n0, n1, n2 = o.n
    eps = 1e-3
    y = o.zeros()
    y[12 * T:13 * T] = 1.0
    y[23 * T:24 * T] = 1.0
    y[19 * T:20 * T] = bz
    K = (eps * (-1.0) ** np.arange(n2))[:, None, None] * np.ones((n2, n1, n0))
    y[13 * T:14 * T] = K.reshape(-1)
    r = o.rhs(y)
    m = o.interior_mask()
    Kv = y[13 * T:14 * T][m]
    adv = r[13 * T:14 * T][m] - Kv * Kv / 3.0
    # damping at every interior point, at a rate of order |beta| / (grid spacing)
    assert np.all(adv * Kv < 0.0)
    assert np.min(-adv / Kv) > 0.1
