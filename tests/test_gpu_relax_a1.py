"""The homogeneous relaxation of viscous stress and heat flux of Sec. 5.A.1
(Grad-17 initial state, N2 at 4000 K, n = 1e24 m^-3, Z_rot = 10, Z_vib = 50)
through the library with both methods, 2e6 particles: the normalized L2 errors
against the analytic relaxation (App. B) reproduce the pattern of the paper's
tables tab:L2norm_sigma and tab:L2norm_q (printed for 1e7 particles):
  stress, FPM      0.013 0.082 0.209 0.874   at dt/tau_c = 0.1 0.5 1 2
  stress, USP-FPM  0.007 0.008 0.037 0.256
  heat fluxes: FPM <= 0.021 at every dt; USP-FPM <= 0.027 up to dt = tau_c and
  0.108 - 0.117 at dt = 2 tau_c.
The bars allow for the noise of 2e6 particles (about 0.02 on these errors)."""
import pytest

from paper_2508_05642_gb300 import run_relax, usp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def res():
    return run_relax.run(N=2_000_000, precision=usp.USP_FP32, seed=2)["runs"]


def test_fpm_stress_error_is_first_order(res):
    e = [res["FPM"][k]["sigma"] for k in ("0.1", "0.5", "1", "2")]
    assert e[0] < 0.045
    assert 0.06 < e[1] < 0.11
    assert 0.17 < e[2] < 0.27
    assert 0.75 < e[3] < 1.0


def test_usp_stress_error_stays_small_to_one_collision_time(res):
    e = [res["USP-FPM"][k]["sigma"] for k in ("0.1", "0.5", "1", "2")]
    assert e[0] < 0.045 and e[1] < 0.045 and e[2] < 0.08
    assert 0.18 < e[3] < 0.34
    # second order against first: the USP-FPM error is the smaller one from 0.5 on
    for k in ("0.5", "1", "2"):
        assert res["USP-FPM"][k]["sigma"] < 0.6 * res["FPM"][k]["sigma"]


def test_heat_flux_errors(res):
    for k in ("0.1", "0.5", "1", "2"):
        for q in ("q_tr", "q_rot", "q_vib"):
            assert res["FPM"][k][q] < 0.08
            if k != "2":
                assert res["USP-FPM"][k][q] < 0.07
            else:
                assert res["USP-FPM"][k][q] > 0.07
        assert all(res[m][k]["flags"] == 0 for m in ("FPM", "USP-FPM"))
