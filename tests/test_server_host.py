"""The solve server's host-side logic on the CPU (no GPU): FIFO admission
under the device-memory budget, refusal of oversize requests and of work
beyond the queue limit, cancellation before admission, a failing setup
(zero pivot) reported on its own request only, and shutdown.  The host-only
server sets requests up and finishes them with ERR_NO_DEVICE (no solve)."""
import time

import numpy as np
import pytest

import paper_2111_09512_gb300 as silu
import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    silu.build()


def rhs(A):
    return np.ones(len(A[0]) - 1)


def test_requests_flow_through_host_server():
    S = silu.Server(device=-1, hbm_budget=1 << 30, workers=2, max_queue=16)
    systems = [synth.cutcell7(e, seed=e) for e in (6, 9, 4, 12, 7)]
    tickets = []
    for A in systems:
        st, t = S.submit(A, rhs(A))
        assert st == silu.OK
        tickets.append(t)
    for t in tickets:
        done, res, _ = S.poll(t, wait=True, want_x=False)
        assert done and res.status == silu.ERR_NO_DEVICE
        assert res.t_submit <= res.t_admit <= res.t_setup_done <= res.t_done
        assert res.device_bytes > 0
    st = S.stats()
    assert st["completed"] == 5 and st["queued"] == 0 and st["bytes_in_use"] == 0
    with pytest.raises(silu.SiluError):
        S.poll(tickets[0])  # released after it was handed out
    S.close()


def test_budget_refusal_queue_limit_and_fifo_admission():
    A_big = synth.cutcell7(20, seed=1)
    A_small = synth.cutcell7(5, seed=2)
    # a request larger than the whole budget is refused outright
    S = silu.Server(device=-1, hbm_budget=200_000, workers=1, max_queue=2)
    st, _ = S.submit(A_big, rhs(A_big))
    assert st == silu.ERR_OOM
    S.close()
    # one slot, queue of two: the fourth concurrent submission is refused
    S = silu.Server(device=-1, hbm_budget=1 << 30, workers=1, max_queue=2)
    accepted, refused = [], 0
    for k in range(12):
        st, t = S.submit(A_big, rhs(A_big))
        if st == silu.OK:
            accepted.append(t)
        else:
            assert st == silu.ERR_BUSY
            refused += 1
    assert refused > 0 and S.stats()["refused"] == refused
    admits = []
    for t in accepted:
        done, res, _ = S.poll(t, wait=True, want_x=False)
        admits.append(res.t_admit)
    assert admits == sorted(admits)  # first in, first admitted
    S.close()


def test_cancel_before_admission_and_failing_setup():
    S = silu.Server(device=-1, hbm_budget=1 << 30, workers=1, max_queue=32)
    A = synth.cutcell7(24, seed=3)
    first = [S.submit(A, rhs(A))[1] for _ in range(3)]
    st, victim = S.submit(A, rhs(A))
    assert st == silu.OK
    assert S.cancel(victim) == silu.OK
    # a singular system: its setup fails, the others are unaffected
    bad = (np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.int32), np.array([0.0, 1.0, 1.0, 2.0]))
    st, tb = S.submit(bad, np.ones(2))
    assert st == silu.OK
    done, res, _ = S.poll(victim, wait=True, want_x=False)
    assert res.status == silu.ERR_CANCELLED
    done, res, _ = S.poll(tb, wait=True, want_x=False)
    assert res.status == silu.ERR_ZERO_PIVOT
    for t in first:
        done, res, _ = S.poll(t, wait=True, want_x=False)
        assert res.status == silu.ERR_NO_DEVICE
    S.close()


def test_shutdown_cancels_waiting_requests():
    S = silu.Server(device=-1, hbm_budget=1 << 30, workers=1, max_queue=64)
    A = synth.cutcell7(40, seed=4)
    tickets = [S.submit(A, rhs(A))[1] for _ in range(6)]
    time.sleep(0.05)
    S.close()  # running request completes, waiting ones are cancelled; no hang
