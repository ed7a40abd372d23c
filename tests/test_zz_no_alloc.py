"""The allocation-free statistics entry point, checked against lb_ch_observe.

lb_ch_field_stats_noalloc exists for callers that may not allocate device memory (code that runs while
another framework owns the memory pool, or plugins restricted to the buffers they are given): it keeps
its partial sums in a fixed device array of the library instead of allocating scratch.  This file runs
last so that a failure here leaves every other test already run.  The device buffers below are the
test's own (allocated with torch); the entry point itself allocates nothing.
"""
import math

import numpy as np
import pytest

from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(p, phi0, nsteps):
    with abi.Simulation(p, phi0, prec="f64") as sim:
        sim.step(nsteps)
        phi = sim.phi()
        ref = {w: sim.observe(w) for w in (abi.LBCH_OBS_MASS, abi.LBCH_OBS_ERR_L2, abi.LBCH_OBS_MAX,
                                           abi.LBCH_OBS_MIN)}
    return phi, ref


def _noalloc(phi, phi0, pad=0):
    dev = torch.device("cuda", torch.cuda.current_device())
    ny, nx = phi.shape
    pitch = nx + pad
    a = np.zeros((ny, pitch)); a[:, :nx] = phi
    b = np.zeros((ny, pitch)); b[:, :nx] = phi0
    d_phi = torch.from_numpy(a).to(dev)
    d_phi0 = torch.from_numpy(b).to(dev)
    out = torch.full((6,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    abi.lb_ch_field_stats_noalloc(d_phi.data_ptr(), d_phi0.data_ptr(), nx, ny, pitch, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def _check(o, ref):
    tol = 1e-12  # the FP64 parity tolerance; only the order of the sums differs
    assert abs(o[0] - ref[abi.LBCH_OBS_MASS]) <= tol * abs(ref[abi.LBCH_OBS_MASS])
    assert abs(math.sqrt(o[1] / o[2]) - ref[abi.LBCH_OBS_ERR_L2]) <= tol * ref[abi.LBCH_OBS_ERR_L2]
    assert o[3] == ref[abi.LBCH_OBS_MAX] and o[4] == ref[abi.LBCH_OBS_MIN]
    assert o[5] == 0.0


def test_noalloc_matches_observe_on_two_calls_in_a_row():
    p, phi0, _ = wl.zalesak(n=96)
    phi, ref = _reference(p, phi0, 150)
    first = _noalloc(phi, phi0)
    _check(first, ref)
    second = _noalloc(phi, phi0)          # the shared partials array is reused
    _check(second, ref)
    assert np.array_equal(first, second)  # same blocks, same order: the same bits


def test_noalloc_other_size_and_pitch_after_a_larger_call():
    p, phi0, _ = wl.single_vortex(n=512, T=100)
    phi_big, ref_big = _reference(p, phi0, 20)
    _check(_noalloc(phi_big, phi0), ref_big)
    q, f0, _ = wl.translation(nx=40)
    phi_small, ref_small = _reference(q, f0, 30)
    _check(_noalloc(phi_small, f0, pad=24), ref_small)  # fewer blocks than the previous call


def test_noalloc_rejects_bad_arguments():
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    out = torch.zeros(6, dtype=torch.float64, device=dev)
    cases = [((buf.data_ptr(), buf.data_ptr(), 1 << 16, 1 << 16, 1 << 16), "maximum"),  # too many nodes
             ((buf.data_ptr(), buf.data_ptr(), 4, 4, 3), "pitch"),                       # pitch < nx
             ((0, buf.data_ptr(), 4, 4, 4), "device pointers")]                          # NULL field
    for args, words in cases:
        with pytest.raises(abi.LbchError) as ei:
            abi.lb_ch_field_stats_noalloc(*args, out.data_ptr(), 0)
        assert ei.value.status == abi.LBCH_EINVAL
        assert words in str(ei.value)


def test_noalloc_counts_non_finite_values_and_leaves_them_out():
    p, phi0, _ = wl.zalesak(n=64)
    phi, _ = _reference(p, phi0, 40)
    bad = phi.copy()
    rng = np.random.default_rng(7)
    idx = rng.choice(bad.size, size=13, replace=False)
    vals = [np.nan, np.inf, -np.inf]
    for k, i in enumerate(idx):
        bad.flat[i] = vals[k % 3]
    o = _noalloc(bad, phi0, pad=8)
    keep = np.isfinite(bad)
    assert o[5] == 13.0
    tol = 1e-12
    assert abs(o[0] - bad[keep].sum()) <= tol * abs(bad[keep].sum())
    d = (bad - phi0)[keep]
    assert abs(o[1] - float((d * d).sum())) <= tol * float((d * d).sum())
    assert abs(o[2] - float((phi0[keep] ** 2).sum())) <= tol * float((phi0[keep] ** 2).sum())
    assert o[3] == bad[keep].max() and o[4] == bad[keep].min()
    # the next call on a clean field is unaffected by the shared scratch of this one
    _check(_noalloc(phi, phi0), {abi.LBCH_OBS_MASS: float(phi.sum()),
                                 abi.LBCH_OBS_ERR_L2: float(np.sqrt(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum())),
                                 abi.LBCH_OBS_MAX: float(phi.max()), abi.LBCH_OBS_MIN: float(phi.min())})


_THREADED = r"""
import sys, threading
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl
p, phi0, _ = wl.zalesak(n=64)
with abi.Simulation(p, phi0, prec="f64") as sim:
    sim.step(20)
    phi = sim.phi()
    mass = sim.observe(abi.LBCH_OBS_MASS)
dev = torch.device("cuda", 0)
d_phi = torch.from_numpy(phi).to(dev)
d_phi0 = torch.from_numpy(phi0).to(dev)
outs = [torch.full((6,), float("nan"), dtype=torch.float64, device=dev) for _ in range(8)]
streams = [torch.cuda.Stream(device=dev) for _ in range(8)]
torch.cuda.synchronize()
errors = []
go = threading.Barrier(8)
def work(k):
    try:
        go.wait()  # every thread makes its first call at once
        abi.lb_ch_field_stats_noalloc(d_phi.data_ptr(), d_phi0.data_ptr(), 64, 64, 64, outs[k].data_ptr(),
                                      streams[k].cuda_stream)
        streams[k].synchronize()
    except Exception as e:
        errors.append(repr(e))
threads = [threading.Thread(target=work, args=(k,)) for k in range(8)]
for t in threads: t.start()
for t in threads: t.join()
assert not errors, errors
# the calls ran on different streams and shared the scratch array, so they may have raced (as documented);
# one more call alone must give the right answer
out = torch.full((6,), float("nan"), dtype=torch.float64, device=dev)
abi.lb_ch_field_stats_noalloc(d_phi.data_ptr(), d_phi0.data_ptr(), 64, 64, 64, out.data_ptr(), 0)
torch.cuda.synchronize()
o = out.cpu().numpy()
assert abs(o[0] - mass) <= 1e-12 * abs(mass) and o[5] == 0.0, o
print("ok")
"""


def test_noalloc_first_calls_from_several_threads_at_once(tmp_path):
    """The first calls in a fresh process, from eight host threads at once, all set up the scratch address
    without error (the per-context cache is filled under a lock), and the next call is correct."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "threaded.py"
    script.write_text(_THREADED)
    r = subprocess.run([sys.executable, str(script), root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
