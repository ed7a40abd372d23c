"""The binomial (revolve) schedule of the checkpointed reverse sweep, checked on the CPU against a model of
the device: it must hand every adjoint step the forward phi of its own step, in reverse order, once; keep at
most `checkpoints` stored states besides the initial one; and, with one-step leaves, run exactly the minimal
number of forward steps, which a brute-force recursion over every split point gives here."""
import functools

import pytest

pytest.importorskip("torch")
from paper_1805_00007_gb300.autograd import revolve_schedule  # noqa: E402


def _replay(T, acts):
    """Execute the actions on a model whose state is the step index; returns the sweeps in order and the
    forward steps taken."""
    cur, slots, tape, sweeps, fwd = 0, {0: 0}, None, [], 0
    for a in acts:
        if a[0] == "advance":
            cur += a[1]
            fwd += a[1]
        elif a[0] == "save":
            slots[a[1]] = cur
        elif a[0] == "load":
            cur = slots[a[1]]
        elif a[0] == "free":
            del slots[a[1]]
        elif a[0] == "tape":
            assert a[1] == cur, "a tape starts from the state it records"
            tape = list(range(cur, cur + a[2]))
            cur += a[2]
            fwd += a[2]
        elif a[0] == "sweep":
            assert tape == list(range(a[1], a[1] + a[2])), "a sweep consumes the tape of its own steps"
            sweeps.extend(range(a[1] + a[2] - 1, a[1] - 1, -1))
        assert cur <= T
    return sweeps, fwd


@functools.lru_cache(maxsize=None)
def _optimal(n, s):
    """Least forward steps (the taped one of each step included) to reverse n steps from a stored start
    state with s free slots."""
    if n == 1:
        return 1
    if s == 0:
        return n * (n + 1) // 2
    return min(m + _optimal(n - m, s - 1) + _optimal(m, s) for m in range(1, n))


@pytest.mark.parametrize("T", [1, 2, 7, 13, 40, 97])
@pytest.mark.parametrize("snaps", [0, 1, 2, 4])
@pytest.mark.parametrize("leaf", [1, 3, 8])
def test_schedule_reverses_every_step_once(T, snaps, leaf):
    acts, st = revolve_schedule(T, snaps, leaf)
    sweeps, fwd = _replay(T, acts)
    assert sweeps == list(range(T - 1, -1, -1))
    assert fwd == st["forward_steps"]
    assert st["slots"] <= snaps + 1


@pytest.mark.parametrize("snaps", [0, 1, 2, 3, 4])
def test_one_step_leaves_are_optimal(snaps):
    for T in range(1, 41):
        _, st = revolve_schedule(T, snaps, 1)
        assert st["forward_steps"] == _optimal(T, snaps), (T, snaps)


def test_single_vortex_schedule():
    """The 8000-step single-vortex reverse sweep with 16 stored states and tapes of 64 steps: 125 leaves,
    repetition number 3 (C(19, 17) = 171 >= 125 > C(18, 17)), under three times the run's length in forward
    steps, the first forward pass included."""
    _, st = revolve_schedule(8000, 16, 64)
    assert st["repetitions"] == 3 and st["slots"] <= 17
    assert st["forward_steps"] < 3 * 8000
