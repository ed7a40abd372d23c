"""Parameter sweeps of the paper's accuracy tests, every parameter point an instance of one ensemble.

The ensemble path advances all instances together (one launch per step), so a sweep over tau_g, the
model and the Peclet number costs about one run of the largest instance.  The error is Eq. err,
||E_phi||_2 = sqrt(sum (phi(T) - phi(0))^2 / sum phi(0)^2), reduced on the GPU in FP64.
"""
from __future__ import annotations

import math

from . import abi
from . import workloads as wl

TAU_STAR = 0.5 + math.sqrt(3) / 6  # K = 0 (Remark I)


def _run(setups, nsteps: int, prec: str, stream=None) -> list[float]:
    params, fields = zip(*setups)
    with abi.Simulation(list(params), list(fields), prec=prec, stream=stream) as sim:
        sim.step(nsteps)
        return [float(e) for e in sim.observe_all(abi.LBCH_OBS_ERR_L2)]


def translation_tau_sweep(taus, models=(1, 2), L0: int = 200, prec: str = "f32", periods: int = 1,
                          U0: float = 0.02, Pe: float = 200.0, W: float = 2.0, rho_ratio: float = 2.0,
                          stream=None) -> dict:
    """Error of the diagonal translation (Sec. III.A: R = L0/5, u = (U0, U0), phiA = -phiB = 1,
    sigma = 0.01) after `periods` periods T = L0/U0, for every (tau_g, model) pair."""
    keys, setups = [], []
    for tau in taus:
        for model in models:
            p, phi0, T = wl.paper_translation(L0=L0, U0=U0, Pe=Pe, W=W, tau=tau, rho_ratio=rho_ratio, model=model)
            keys.append((tau, model))
            setups.append((p, phi0))
    return dict(zip(keys, _run(setups, periods * T, prec, stream)))


def translation_pe_sweep(pes, models=(1, 2), L0: int = 200, prec: str = "f32", tau: float = 1.0,
                         stream=None) -> dict:
    """Error of the diagonal translation after one period for every (Pe, model) pair (the Peclet-number
    study of Sec. III.A)."""
    keys, setups = [], []
    for pe in pes:
        for model in models:
            p, phi0, T = wl.paper_translation(L0=L0, Pe=pe, tau=tau, rho_ratio=2.0, model=model)
            keys.append((pe, model))
            setups.append((p, phi0))
    return dict(zip(keys, _run(setups, T, prec, stream)))
