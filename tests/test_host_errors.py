"""Refusals that the library makes on the host, before any device work (CPU).

A run is refused when a pointer table or pointer is NULL (HFAV_EINVAL), when
a pointer is not 16-byte aligned (HFAV_EALIGN), when a goal aliases an axiom
it is not declared to alias (HFAV_EINVAL) and when n_steps is not positive;
the allocation-free chain refuses arrays that overlap.  None of these reach
the GPU: the pointers below are never dereferenced.  The HFAV_SCHEDULE
environment variable overrides a NULL / "auto" schedule argument.
"""
import ctypes

import pytest

from paper_1710_08774_gb300 import hfav as H

EINVAL, EALIGN = -1, -6


def _plan():
    return H.Plan(H.chain2d_dag(), [H.Grid.make((64, 48), (1, 68), 2)], H.HFAV_F64, H.HFAV_BC_PERIODIC,
                  "sweep:reg:32x4")


def _run(P, a, g, n_steps=1):
    at = (ctypes.c_void_p * 1)(a)
    gt = (ctypes.c_void_p * 1)(g)
    return H.load().hfav_run(P.h, at, gt, n_steps, None)


def test_null_pointers_refused():
    P = _plan()
    assert _run(P, None, 0x20000) == EINVAL
    assert b"null axiom" in H.load().hfav_last_error()
    assert _run(P, 0x10000, None) == EINVAL
    assert b"null goal" in H.load().hfav_last_error()
    assert H.load().hfav_run(P.h, None, None, 1, None) == EINVAL


def test_misaligned_pointers_refused():
    P = _plan()
    assert _run(P, 0x10008, 0x20000) == EALIGN
    assert _run(P, 0x10000, 0x20004) == EALIGN
    assert b"16-byte" in H.load().hfav_last_error()


def test_undeclared_alias_and_steps_refused():
    P = _plan()
    assert _run(P, 0x10000, 0x10000) == EINVAL
    assert b"dag.inout" in H.load().hfav_last_error()
    assert _run(P, 0x10000, 0x20000, n_steps=0) == EINVAL
    assert _run(P, 0x10000, 0x20000, n_steps=2) == EINVAL   # no feedback: one step only


@pytest.mark.parametrize("delta", [0, 8 * 1, 8 * 67, -8 * 5])
def test_static_chain_refuses_overlap(delta):
    # (48 + 4) rows of pitch 68 doubles: any start within that span overlaps
    base = 1 << 32
    rc = H.load().hfav_chain2d_static(ctypes.c_void_p(base), 64, 48, 68, 2, H.HFAV_BC_PERIODIC, None,
                                      ctypes.c_void_p(base + delta), None)
    assert rc == EINVAL
    assert b"overlap" in H.load().hfav_last_error()


def test_schedule_environment_override(monkeypatch):
    g = [H.Grid.make((64, 48), (1, 68), 2)]
    monkeypatch.setenv("HFAV_SCHEDULE", "full:smem:64x4")
    assert H.Plan(H.chain2d_dag(), g, H.HFAV_F64).schedule == "full:smem:64x4"
    # an explicit argument wins over the environment
    assert H.Plan(H.chain2d_dag(), g, H.HFAV_F64, schedule="unfused").schedule.startswith("unfused")
    monkeypatch.setenv("HFAV_SCHEDULE", "tuned")
    assert H.Plan(H.chain2d_dag(), g, H.HFAV_F64).schedule == H.Plan(H.chain2d_dag(), g, H.HFAV_F64,
                                                                     schedule="auto").schedule
    monkeypatch.setenv("HFAV_SCHEDULE", "sideways")
    with pytest.raises(H.HfavError) as e:
        H.Plan(H.chain2d_dag(), g, H.HFAV_F64)
    assert e.value.code == EINVAL


@pytest.mark.parametrize("cap", [0, 11, 2.5])
def test_newton_cap_out_of_range_refused(cap):
    with pytest.raises(H.HfavError):
        H.Plan(H.godunov_dag(newton_max=cap), [H.Grid.make((64, 48), (1, 64), 0)], H.HFAV_F64, H.HFAV_BC_PERIODIC)
