"""The GWR/MPR finding of the GPU experiment reproduced by the oracle at a small size (Sec. 4,
Fig. mu; Sec. 5, Fig. res). The same isotropic model is fitted to the same anisotropic
target data. At a strong regularisation weight the global entropy holds the fit well above
chi^2/J = 1, and the moving priors reach about 1. The MPR weights also scatter less about
their cell means. This shows the finding belongs to the method, not to the GPU code."""
import oracle as O
from paper_1202_2355_gb300 import gwr_vs_mpr as X


def _fit(mode, wl, targets, mu, steps):
    obs, Y, sig = targets
    run = O.Run(wl.potential, obs, Y, sig, dict(wl.prior, mode=mode), dict(wl.params, mu=mu), wl.model)
    assert run.step(steps) == 0
    ws, wd, cnt = O.grid_weights(wl.potential, wl.prior, run.ps)
    return run.chi2 / len(Y), O.weight_rms(wd, cnt, 50) * len(run.w) / ws.sum()


def test_mpr_fits_and_smooths_where_gwr_does_not():
    O.build()
    wl = X.workload(20_000, 200_000)
    targets = O.from_workload(wl)
    c_gwr, r_gwr = _fit("gwr", wl, targets, 1e5, 1000)
    c_mpr, r_mpr = _fit("mpr", wl, targets, 1e5, 1000)
    assert c_gwr > 2.5 and c_mpr < 1.6 and c_gwr > 2.5 * c_mpr, (c_gwr, c_mpr)
    assert r_mpr < 0.8 * r_gwr, (r_gwr, r_mpr)
