"""GWR against MPR on a radially anisotropic target (Sec. 4, Fig. mu; Sec. 5, Fig. res),
at a reduced size, through the library. Two findings of the paper that hold in this
synthetic setup are asserted. At a regularisation weight where the global entropy
already spoils the fit (chi^2/J > 1), the moving priors still fit the data (chi^2/J < 1).
The MPR model is also smoother: a smaller rms of the weights about their cell means.
The grid-less variant (window priors, Sec. 7) recovers the target's (E, x) masses better than
the initial model and than the cell priors (lower Delta_grid) and keeps the fit."""
import pytest

from paper_1202_2355_gb300 import gwr_vs_mpr as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()


def test_mpr_fits_where_gwr_does_not_and_is_smoother():
    init, gwr, mpr, mprw = list(X.scan(300_000, 1_000_000, 10_000, [1e5], modes=("gwr", "mpr", "mprw")))
    assert init["mode"] == "initial" and init["chi2_per_J"] > 10
    assert gwr["mode"] == "gwr" and mpr["mode"] == "mpr" and mprw["mode"] == "mprw"
    assert gwr["chi2_per_J"] > 1.5, gwr
    assert mpr["chi2_per_J"] < 0.6, mpr
    assert mpr["weight_rms_rel"] < 0.5 * gwr["weight_rms_rel"]
    # both fits move the model towards the target's kinematics
    assert gwr["delta_kin"] < init["delta_kin"] and mpr["delta_kin"] < init["delta_kin"]
    # the window priors fit, and lower Delta_grid below the initial model's and MPR's
    assert mprw["chi2_per_J"] < 1.0, mprw
    assert mprw["delta_grid"] < 0.9 * init["delta_grid"] and mprw["delta_grid"] < 0.8 * mpr["delta_grid"], \
        (init["delta_grid"], mpr["delta_grid"], mprw["delta_grid"])
    assert mprw["delta_kin"] < init["delta_kin"]
