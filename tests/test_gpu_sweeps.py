"""The batched parameter sweeps (paper_1805_00007_gb300.sweeps) on the GPU against the oracle, and the
paper's relaxation-time claims of Sec. III.A on the GPU results."""
import math

import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import sweeps
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,rtol", [("f64", 1e-10), ("f32", 1e-4)])
def test_tau_sweep_matches_oracle_and_paper(prec, rtol):
    taus = (0.6, sweeps.TAU_STAR, 1.0, 1.3)
    got = sweeps.translation_tau_sweep(taus, models=(1, 2, 3), L0=50, prec=prec)
    for (tau, model), e in got.items():
        p, phi0, T = wl.paper_translation(L0=50, tau=tau, rho_ratio=2.0, model=model)
        phi, _ = oracle.simulate(p, phi0, T)
        ref = oracle.observe(phi, phi0)["err_l2"]
        assert abs(e - ref) <= rtol * ref, (tau, model, e, ref)
    star = sweeps.TAU_STAR
    assert all(got[star, 1] < got[t, 1] for t in taus if t != star)
    assert all(got[t, 2] < 0.7 * got[t, 1] for t in taus if t != star)


def test_pe_sweep_runs_as_one_ensemble():
    got = sweeps.translation_pe_sweep((50.0, 200.0, 1000.0), models=(1, 2), L0=50, prec="f64")
    for (pe, model), e in got.items():
        p, phi0, T = wl.paper_translation(L0=50, Pe=pe, tau=1.0, rho_ratio=2.0, model=model)
        phi, _ = oracle.simulate(p, phi0, T)
        assert abs(e - oracle.observe(phi, phi0)["err_l2"]) <= 1e-10 * e
