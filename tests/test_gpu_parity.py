"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (max |phi_gpu - phi_oracle| over every node):
  FP64 path: 1e-12  (the same arithmetic in a different order, with explicit fused multiply-adds)
  FP32 path: 1e-5   (single-precision state and arithmetic; the velocity tables are built in double)
  F16S path: 2e-3 after 50 steps (half-precision populations; rounding of 2^-11 relative per step on
             populations of size up to ~0.15, random-walk accumulated) -- see test_f16s_parity
Sizes span several tiles of every kernel form (row-sweep strips of 56 columns, tiles of 32 x 16 and
32 x 8) with ragged tails in both directions.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _gpu(p, phi0, nsteps, prec):
    with abi.Simulation(p, phi0, prec=prec) as sim:
        sim.step(nsteps)
        return sim.phi()


def _maxdiff(a, b):
    return float(np.max(np.abs(a - b)))


def _cases():
    n = 0
    out = []
    for vel in (wl.VEL_UNIFORM, wl.VEL_ROTATION, wl.VEL_VORTEX, wl.VEL_REV_SHEAR, wl.VEL_DEFORM, wl.VEL_SHEAR):
        for model in (1, 2):
            n += 1
            out.append((vel, model, n))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("vel,model,seed", _cases())
def test_small_grids_every_flow(prec, vel, model, seed):
    nx, ny = 45, 37  # two tiles + ragged tail in x; several tiles + tail in y
    walls = 1 if vel == wl.VEL_SHEAR else 0
    p = wl.make_params(nx=nx, ny=ny, vel=vel, walls=walls, model=model, U0=0.03, ux0=0.03, uy0=-0.02,
                       xc=22.0, yc=18.0, half=22.0, Tper=30.0, shear=2e-3, tau=0.85, M=0.02,
                       sigma=0.02, W=3.0, rhoB=0.4, nvort=2)
    phi0 = np.clip(wl.random_smooth_phi(nx, ny, seed) + 0.6 * wl.circle_phi(nx, ny, 20.3, 17.7, 9.0, 3.0) - 0.3,
                   -0.2, 1.2)
    nsteps = 50  # crosses the reversal time of the reversing shear
    ref, _ = oracle.simulate(p, phi0, nsteps)
    got = _gpu(p, phi0, nsteps, prec)
    assert _maxdiff(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_zero_steps_is_initial_field(prec):
    p, phi0, _ = wl.zalesak(n=40)
    got = _gpu(p, phi0, 0, prec)
    assert _maxdiff(got, phi0) <= (0.0 if prec == "f64" else 1e-7)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 7), (33, 4), (4, 41), (64, 16), (31, 9)])
def test_tiny_and_ragged_sizes(prec, nx, ny):
    p = wl.make_params(nx=nx, ny=ny, vel=wl.VEL_ROTATION, U0=0.02, xc=nx / 2, yc=ny / 2, half=max(nx, ny) / 2,
                       tau=1.0, M=0.02, sigma=0.02, W=3.0)
    phi0 = wl.random_smooth_phi(nx, ny, seed=nx * 100 + ny)
    ref, _ = oracle.simulate(p, phi0, 25)
    assert _maxdiff(_gpu(p, phi0, 25, prec), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_translation_full_period(prec):
    """The 100 x 100 diagonal translation for its whole period (2500 steps, CUDA graphs + tail steps)."""
    p, phi0, T = wl.translation()
    ref, _ = oracle.simulate(p, phi0, T)
    with abi.Simulation(p, phi0, prec=prec) as sim:
        sim.step(T)
        got = sim.phi()
        err = sim.observe(abi.LBCH_OBS_ERR_L2)
        mass = sim.observe(abi.LBCH_OBS_MASS)
        mx, mn = sim.observe(abi.LBCH_OBS_MAX), sim.observe(abi.LBCH_OBS_MIN)
    assert _maxdiff(got, ref) <= TOL[prec]
    ob = oracle.observe(ref, phi0)
    assert abs(err - ob["err_l2"]) <= 0.01 * ob["err_l2"]
    assert abs(mx - ob["max"]) <= TOL[prec] and abs(mn - ob["min"]) <= TOL[prec]
    rel_mass = abs(mass - phi0.sum()) / phi0.sum()
    assert rel_mass <= (1e-13 if prec == "f64" else 1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_zalesak_full_grid(prec):
    """256 x 256 Zalesak grid (the benchmark's launch configuration) for 200 steps."""
    p, phi0, _ = wl.zalesak()
    ref, _ = oracle.simulate(p, phi0, 200)
    assert _maxdiff(_gpu(p, phi0, 200, prec), ref) <= TOL[prec]


def test_single_vortex_full_grid():
    p, phi0, _ = wl.single_vortex()
    ref, _ = oracle.simulate(p, phi0, 30)
    for prec in ("f64", "f32"):
        assert _maxdiff(_gpu(p, phi0, 30, prec), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_ensemble_matches_each_instance(prec):
    """An ensemble of instances of different sizes and parameters in one launch equals each instance
    simulated alone by the oracle."""
    ens = wl.shear_ensemble(n_inst=7, sides=(16, 37, 64, 20), seed=5)
    # make the shear visible at these small sizes
    ens = [(dict(p, shear=p["shear"] * 40.0, Ustar=p["Ustar"] * 40.0), f) for p, f in ens]
    params, fields = zip(*ens)
    nsteps = 70
    with abi.Simulation(list(params), list(fields), prec=prec) as sim:
        sim.step(nsteps)
        got = [sim.phi(k) for k in range(len(params))]
        masses = sim.observe_all(abi.LBCH_OBS_MASS)
    for k, (p, f) in enumerate(ens):
        ref, _ = oracle.simulate(p, f, nsteps)
        assert _maxdiff(got[k], ref) <= TOL[prec], k
        assert abs(masses[k] - f.sum()) <= (1e-12 if prec == "f64" else 1e-4) * f.sum()


def test_observables_match_oracle_definition():
    p, phi0, _ = wl.zalesak(n=96)
    ref, _ = oracle.simulate(p, phi0, 120)
    ob = oracle.observe(ref, phi0)
    with abi.Simulation(p, phi0, prec="f64") as sim:
        sim.step(120)
        assert abs(sim.observe(abi.LBCH_OBS_MASS) - ob["mass"]) <= 1e-11
        assert abs(sim.observe(abi.LBCH_OBS_ERR_L2) - ob["err_l2"]) <= 1e-11
        assert abs(sim.observe(abi.LBCH_OBS_MAX) - ob["max"]) <= 1e-12
        assert abs(sim.observe(abi.LBCH_OBS_MIN) - ob["min"]) <= 1e-12
        assert sim.observe(abi.LBCH_OBS_STEP) == 120
        # reductions are deterministic: a second call gives the same bits
        a = sim.observe(abi.LBCH_OBS_ERR_L2)
        assert a == sim.observe(abi.LBCH_OBS_ERR_L2)


def test_f16s_parity():
    """Shifted half storage: phi in float, g_1..g_8 in half, g_0 implied by phi."""
    p, phi0, _ = wl.zalesak(n=96)
    ref, _ = oracle.simulate(p, phi0, 50)
    with abi.Simulation(p, phi0, prec="f16s") as sim:
        sim.step(50)
        got = sim.phi()
        mass = sim.observe(abi.LBCH_OBS_MASS)
    assert _maxdiff(got, ref) <= 2e-3
    assert abs(mass - phi0.sum()) <= 1e-5 * phi0.sum()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_steps_split_across_calls_equal_one_call(prec):
    """Graph replays (of 512 and of 64 steps), single launches and their mix advance the same state, bit for
    bit, and the time-dependent flow sees the right step index throughout (FP32 at 64^2 runs the two-step
    kernel, FP64 a one-step form)."""
    p, phi0, _ = wl.single_vortex(n=64, T=400)
    with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(p, phi0, prec=prec) as b:
        a.step(131)
        for k in (1, 64, 3, 63):
            b.step(k)
        assert np.array_equal(a.phi(), b.phi())
        a.step(1150)  # two graphs of 512, two of 64, then single launches
        for k in (600, 37, 513):
            b.step(k)
        assert a.observe(abi.LBCH_OBS_STEP) == b.observe(abi.LBCH_OBS_STEP) == 1281
        assert np.array_equal(a.phi(), b.phi())


def test_nonfinite_is_reported():
    """A state that blows up (tau close to 1/2, huge velocity) is reported as LBCH_ENONFINITE."""
    p = wl.make_params(nx=16, ny=16, vel=wl.VEL_UNIFORM, ux0=3.0, uy0=3.0, tau=0.5001, M=1.0, sigma=1.0, W=1.0)
    phi0 = wl.random_smooth_phi(16, 16, seed=1, amp=2.0)
    with abi.Simulation(p, phi0, prec="f64") as sim:
        sim.step(400)
        with pytest.raises(abi.LbchError) as ei:
            sim.observe(abi.LBCH_OBS_MASS)
        assert ei.value.status == abi.LBCH_ENONFINITE


@pytest.mark.parametrize("prec,nshapes,tile,general", [("f64", 5, 1, 1), ("f32", 4, 1, 1), ("f16s", 4, 1, 1),
                                                      ("f64", 5, 1, 0), ("f32", 4, 1, 0),
                                                      ("f64", 4, 0, 1), ("f32", 4, 0, 1), ("f16s", 4, 0, 1),
                                                      ("f64", 4, 0, 0), ("f32", 4, 0, 0), ("f16s", 4, 0, 0)])
def test_every_tile_shape_gives_the_same_bits(prec, nshapes, tile, general):
    """The result does not depend on the tile shape (each node's arithmetic is the same; only the halo
    overlap between tiles changes), so every shape must reproduce the same bits; the autotuner then
    only picks among equivalent kernels.  Every kernel form: the tile kernel, and the row sweep with
    and without the populations."""
    ens = wl.shear_ensemble(n_inst=3, sides=(37, 64, 16), seed=9)
    params, fields = zip(*ens)
    p, phi0, _ = wl.single_vortex(n=96, T=50)
    outs = []
    for k in range(nshapes):
        with abi.Simulation(p, phi0, prec=prec) as sim, abi.Simulation(list(params), list(fields), prec=prec) as ens_sim:
            for h in (sim.h, ens_sim.h):
                abi.lb_ch_test_hook(h, abi.LBCH_HOOK_TILE_KERNEL, tile)
                abi.lb_ch_test_hook(h, abi.LBCH_HOOK_GENERAL_PATH, general)
                abi.lb_ch_test_hook(h, abi.LBCH_HOOK_TILE_SHAPE, k)
            sim.step(70)
            ens_sim.step(70)
            outs.append([sim.phi()] + [ens_sim.phi(i) for i in range(3)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec,tau", [("f32", 1.0), ("f64", 1.0), ("f16s", 1.0), ("f32", 0.8), ("f16s", 0.8)])
def test_tune_keeps_the_state(prec, tau):
    """The autotuner chooses among kernel forms and shapes that give the same bits, and leaves the state
    where it found it."""
    p, phi0, _ = wl.zalesak(n=128, tau=tau)
    with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(p, phi0, prec=prec, tune=True) as b:
        # row sweep, tile kernel or (periodic, tau_g = 1, not half storage) the two-step kernel
        assert b.tile in ((56, 48), (56, 24), (56, 12), (32, 16), (32, 8), (16, 8), (16, 16), (32, 14))
        assert b.kernel()["threads"] in (64, 128, 256, 512, 768, 1024)
        if prec == "f16s" and tau == 1.0:
            assert b.kernel()["form"] == "sweep_tau1"
        if tau != 1.0:
            assert b.kernel()["form"] != "pair_tau1"
        assert b.observe(abi.LBCH_OBS_STEP) == 0
        a.step(101)  # a graph, then launches of the chosen kernel, and an odd last step
        b.step(101)
        assert np.array_equal(a.phi(), b.phi())


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_kernel_forms_give_the_same_bits(prec):
    """The row sweep with the populations (any tau_g) against the tile kernel, at tau_g = 0.8 and 1.3, for
    a periodic time-dependent flow and for a ragged ensemble with moving walls: the same arithmetic per
    node in another order of work, so the same bits -- on the half-storage path too."""
    for tau in (0.8, 1.3):
        p, phi0, _ = wl.single_vortex(n=96, T=60, tau=tau)
        ens = wl.shear_ensemble(n_inst=3, sides=(37, 64, 16), seed=4, tau=tau)
        ens = [(dict(q, shear=q["shear"] * 30.0, Ustar=q["Ustar"] * 30.0), f) for q, f in ens]
        params, fields = zip(*ens)
        res = []
        for tile in (0, 1):
            with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(list(params), list(fields), prec=prec) as b:
                abi.lb_ch_test_hook(a.h, abi.LBCH_HOOK_TILE_KERNEL, tile)
                abi.lb_ch_test_hook(b.h, abi.LBCH_HOOK_TILE_KERNEL, tile)
                a.step(90)
                b.step(90)
                res.append([a.phi()] + [b.phi(k) for k in range(3)])
        for x, y in zip(res[0], res[1]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_tau1_kernel_equals_general_kernel_bitwise(prec):
    """At tau_g = 1 the populations drop out of Eq. LB (g* = g_eq + S/2).  The row-sweep kernel, which reads
    and writes phi only, must give the same bits as the tile kernel on the general path, which multiplies
    the populations by zero -- for a periodic flow and for a ragged ensemble with moving walls.  On the
    half-storage path the general kernel rounds the streamed populations to half; the sweep keeps them in
    float, so there the two agree to the half rounding only (and the sweep is the closer to the oracle)."""
    p, phi0, _ = wl.single_vortex(n=96, T=60)
    ens = wl.shear_ensemble(n_inst=3, sides=(37, 64, 16), seed=4)
    ens = [(dict(q, shear=q["shear"] * 30.0, Ustar=q["Ustar"] * 30.0), f) for q, f in ens]
    params, fields = zip(*ens)
    res = []
    for general in (0, 1):
        with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(list(params), list(fields), prec=prec) as b:
            abi.lb_ch_test_hook(a.h, abi.LBCH_HOOK_TILE_KERNEL, 0)  # the row sweep
            abi.lb_ch_test_hook(a.h, abi.LBCH_HOOK_GENERAL_PATH, general)
            abi.lb_ch_test_hook(b.h, abi.LBCH_HOOK_GENERAL_PATH, general)
            a.step(90)
            b.step(90)
            res.append([a.phi()] + [b.phi(k) for k in range(3)])
            bytes_lu = a.info()["bytes_per_lu"]
            assert bytes_lu == ({"f64": 160.0, "f32": 88.0, "f16s": 40.0}[prec] if general else
                                {"f64": 16.0, "f32": 16.0, "f16s": 8.0}[prec])
    if prec != "f16s":
        for x, y in zip(res[0], res[1]):
            assert np.array_equal(x, y)
        # the tile kernel drops the populations at tau_g = 1 too: the same bits again
        with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(list(params), list(fields), prec=prec) as b:
            for h in (a.h, b.h):
                abi.lb_ch_test_hook(h, abi.LBCH_HOOK_TILE_KERNEL, 1)
            assert a.kernel()["form"] == "tile_tau1"
            a.step(90)
            b.step(90)
            for x, y in zip([a.phi()] + [b.phi(k) for k in range(3)], res[0]):
                assert np.array_equal(x, y)
    else:
        ref, _ = oracle.simulate(p, phi0, 90)
        assert _maxdiff(res[0][0], ref) <= _maxdiff(res[1][0], ref) + 1e-6
        for x, y in zip(res[0], res[1]):
            assert _maxdiff(x, y) <= 2e-3


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dependent_launch_gives_the_same_bits(prec):
    """Step launches that overlap the previous step's tail (programmatic dependent launch) read the step
    counter and the fields only after that step completes, so they reproduce the plain stream-ordered
    launches bit for bit -- in a time-dependent flow, over graph replays and single launches, at tau_g = 1
    and not."""
    for tau in (1.0, 0.8):
        p, phi0, _ = wl.single_vortex(n=96, T=60, tau=tau)
        out = []
        for no_pdl in (0, 1):
            with abi.Simulation(p, phi0, prec=prec) as sim:
                abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_NO_PDL, no_pdl)
                for k in (64, 5, 128, 1):
                    sim.step(k)
                assert sim.observe(abi.LBCH_OBS_STEP) == 198
                out.append(sim.phi())
        assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16s", 2e-3)])
def test_model3_matches_oracle(prec, tol):
    """Model III (the complete force of Eq. F2-1, time derivatives as one-step backward differences) on a
    periodic time-dependent flow at tau_g = 0.8, 1 (no populations kept) and 1.3, and on a ragged ensemble
    with walls that mixes Models II and III; graph replays and single launches (the stored H crosses both).
    Both kernel forms -- the row sweep (its Model III build, the default) in each of its configurations and
    the tile kernel -- against the oracle and against each other bit for bit (on the half path at tau_g = 1
    the tile kernel streams half-rounded populations, so there the two agree to the tolerance)."""
    nsteps = 131 if prec != "f16s" else 50

    def run(params, fields, form, shape=0):
        with abi.Simulation(params, fields, prec=prec) as sim:
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 1 if form == "tile" else 0)
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_SHAPE, shape)
            assert sim.kernel()["form"] in (("tile", "tile_tau1") if form == "tile" else ("sweep", "sweep_tau1"))
            sim.step(nsteps)
            return [sim.phi(k) for k in range(len(sim.params))]

    for tau in (0.8, 1.0, 1.3):
        p = wl.make_params(nx=45, ny=37, vel=wl.VEL_VORTEX, U0=0.05, Tper=60.0, M=0.02, sigma=0.03, W=3.0,
                           rhoB=0.4, tau=tau, model=3)
        phi0 = np.clip(wl.random_smooth_phi(45, 37, seed=5) + 0.6 * wl.circle_phi(45, 37, 20.0, 18.0, 9.0, 3.0) - 0.3,
                       0, 1)
        ref, _ = oracle.simulate(p, phi0, nsteps)
        with abi.Simulation(p, phi0, prec=prec) as sim:
            assert sim.kernel()["form"] in ("sweep", "sweep_tau1")  # the untuned default
        sweeps = [run(p, phi0, "sweep", k)[0] for k in range(2)]
        tile = run(p, phi0, "tile")[0]
        for got in sweeps + [tile]:
            assert _maxdiff(got, ref) <= tol
        assert np.array_equal(sweeps[0], sweeps[1])
        if not (prec == "f16s" and tau == 1.0):
            assert np.array_equal(sweeps[0], tile)
    ens = wl.shear_ensemble(n_inst=3, sides=(37, 64, 16), seed=6, tau=0.9)
    ens = [(dict(q, shear=q["shear"] * 30.0, Ustar=q["Ustar"] * 30.0, model=3 if k != 1 else 2), f)
           for k, (q, f) in enumerate(ens)]
    params, fields = [q for q, _ in ens], [f for _, f in ens]
    by_form = {form: run(params, fields, form) for form in ("sweep", "tile")}
    for k, (q, f) in enumerate(ens):
        ref, _ = oracle.simulate(q, f, nsteps)
        assert _maxdiff(by_form["sweep"][k], ref) <= tol
        assert np.array_equal(by_form["sweep"][k], by_form["tile"][k])


def test_model3_state_save_load_round_trip():
    """The checkpoint of a Model III handle carries H, so a reloaded state continues bit for bit."""
    torch = pytest.importorskip("torch")
    p = wl.make_params(nx=40, ny=36, vel=wl.VEL_VORTEX, U0=0.05, Tper=50.0, M=0.02, tau=0.8, model=3)
    phi0 = wl.circle_phi(40, 36, 20.0, 18.0, 9.0, 3.0)
    for prec in ("f64", "f32"):
        with abi.Simulation(p, phi0, prec=prec) as sim:
            sim.step(13)
            buf = torch.empty(abi.lb_ch_state_bytes(sim.h), dtype=torch.uint8, device="cuda")
            abi.lb_ch_state_save(sim.h, buf.data_ptr())
            sim.step(70)
            a = sim.phi()
            abi.lb_ch_state_load(sim.h, buf.data_ptr())
            sim.step(70)
            assert np.array_equal(a, sim.phi())


@pytest.mark.parametrize("setup,L0", [("paper_shear_reversal", 64), ("paper_deformation", 80)])
def test_paper_reversing_flows_match_oracle(setup, L0):
    """The paper's reversing shear (Sec. III.C) and deformation (Sec. III.D) workloads at reduced size, over
    their whole return time, every precision against the oracle's final field."""
    p, phi0, N = getattr(wl, setup)(L0=L0)
    ref, _ = oracle.simulate(p, phi0, N)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        with abi.Simulation(p, phi0, prec=prec) as sim:
            sim.step(N)
            assert _maxdiff(sim.phi(), ref) <= tol, prec


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5), ("f16s", 2e-3)])
@pytest.mark.parametrize("form", ["sweep", "tile"])
def test_moving_walls_match_oracle(prec, tol, form):
    """The moving-wall bounce-back (reading R7, pinned on the oracle by the co-moving uniform state) on the
    wall-driven shear case at tau_g = 0.8, where the bounced populations reach phi a step later: every
    kernel form through the C ABI against the oracle.  A wrong sign, factor or a wall at rest moves phi by
    more than 100 times the FP32 tolerance here (tests/test_oracle_pins.py plants each in the oracle)."""
    p, phi0 = wl.moving_wall_case()
    ref, _ = oracle.simulate(p, phi0, 60)
    with abi.Simulation(p, phi0, prec=prec) as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 1 if form == "tile" else 0)
        assert sim.kernel()["form"] == ("tile" if form == "tile" else "sweep")
        sim.step(60)
        assert _maxdiff(sim.phi(), ref) <= tol
    # the co-moving uniform state stays put on the GPU as well
    q = wl.make_params(nx=40, ny=21, walls=1, vel=wl.VEL_UNIFORM, ux0=0.05, uy0=0.0, model=2, tau=0.8, M=0.01)
    with abi.Simulation(q, np.full((21, 40), 0.37), prec=prec) as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 1 if form == "tile" else 0)
        sim.step(70)
        # (the half path rounds the streamed populations; its rest population takes up what they leave, so
        # no phi moves between nodes and the uniform state is kept to float rounding)
        assert _maxdiff(sim.phi(), np.full((21, 40), 0.37)) <= {"f64": 1e-14, "f32": 1e-6, "f16s": 1e-6}[prec]
        assert abs(sim.observe(abi.LBCH_OBS_MASS) - 0.37 * 21 * 40) <= {"f64": 1e-12, "f32": 1e-4, "f16s": 1e-4}[prec]


def test_handles_made_and_freed_reuse_memory_cleanly():
    """Handles take their buffers from a memory pool that keeps freed memory, and their pinned staging from a
    cache: a handle made after others were freed gets memory they wrote.  Every repetition of the same
    sequence of handles (different sizes, precisions, walls, Model III, an ensemble) must give the first
    repetition's results bit for bit."""
    mw, fw = wl.moving_wall_case()
    p3 = wl.make_params(nx=45, ny=37, vel=wl.VEL_VORTEX, U0=0.05, Tper=60.0, M=0.02, sigma=0.03, W=3.0,
                        rhoB=0.4, tau=0.8, model=3)
    f3 = np.clip(wl.random_smooth_phi(45, 37, seed=5) + 0.6 * wl.circle_phi(45, 37, 20.0, 18.0, 9.0, 3.0) - 0.3, 0, 1)
    pz, fz, _ = wl.zalesak(n=96)
    ens = wl.shear_ensemble(n_inst=3, sides=(37, 64, 16), seed=9)
    cases = [(mw, fw, "f32"), (p3, f3, "f64"), (pz, fz, "f16s"), (pz, fz, "f32"),
             ([q for q, _ in ens], [f for _, f in ens], "f32")]
    runs = []
    for rep in range(3):
        out = []
        for p, f, prec in cases:
            with abi.Simulation(p, f, prec=prec) as sim:
                sim.step(23)
                out.append([sim.phi(k) for k in range(len(sim.params))])
        runs.append(out)
    for out in runs[1:]:
        for a, b in zip(runs[0], out):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
