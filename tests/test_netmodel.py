"""The communication model of Pi_MultVerify^R (paper_2411_09287_gb300.netmodel) against the
oracle's ledger, and the trade-off the paper reports for R -- no GPU."""
import hashlib

import numpy as np
import pytest

from oracle import protocols as OP
from oracle import verify as OV
from oracle.shares import Session
from paper_2411_09287_gb300 import netmodel as NM

U64 = np.uint64


@pytest.mark.parametrize("D,R", [(16, 0), (16, 1), (100, 3), (257, 2), (1000, 8), (1024, 5)])
def test_bytes_and_messages_equal_the_oracle_ledger(D, R):
    s = Session(hashlib.sha256(b"netmodel").digest())
    rng = np.random.default_rng(D + R)
    x, y = (rng.integers(0, 2**64, D, dtype=U64) for _ in range(2))
    X, Y = OP.share_input(s, x, 1), OP.share_input(s, y, 2)
    Z = OP.mult(s, X, Y, 3)
    s.ledger.clear()
    assert OV.mult_verify(s, X, Y, Z, 4, R=R)
    assert sum(e.nbytes for e in s.ledger) == NM.verify_bytes(D, R)
    assert len(s.ledger) == NM.verify_messages(R)


def test_dim_after_pads_odd_lengths():
    assert [NM.dim_after(13, r) for r in range(5)] == [13, 7, 4, 2, 1]


@pytest.mark.parametrize("name", ["LAN", "MAN", "WAN"])
def test_larger_batches_want_more_rounds(name):
    net = NM.NETWORKS[name]
    best = [NM.best_R(1 << k, net) for k in (12, 16, 18, 20)]
    assert best == sorted(best) and best[-1] > best[0]


def test_slower_links_want_more_rounds_at_equal_rtt():
    bw = [1e9 / 8, 100e6 / 8, 40e6 / 8, 10e6 / 8]
    best = [NM.best_R(1 << 18, NM.Network(12e-3, b)) for b in bw]
    assert best == sorted(best) and best[-1] > best[0]


def test_longer_round_trips_want_fewer_rounds():
    best = [NM.best_R(1 << 18, NM.Network(rtt, 100e6 / 8)) for rtt in (0.2e-3, 12e-3, 80e-3)]
    assert best == sorted(best, reverse=True) and best[0] > best[-1]


def test_time_at_the_best_R_is_the_minimum():
    net = NM.NETWORKS["MAN"]
    R = NM.best_R(1 << 18, net)
    t = [NM.verify_time(1 << 18, r, net) for r in range(25)]
    assert t[R] == min(t)


def test_best_by_total_adds_measured_computation():
    """With computation that grows with R, the optimum moves to fewer rounds than the
    communication-only optimum; with none it is the communication-only optimum."""
    from paper_2411_09287_gb300 import netrun as NR
    D, net = 1 << 18, NM.NETWORKS["MAN"]
    free = {R: 0.0 for R in range(17)}
    assert NR.best_by_total(free, D, net)[0] == NM.best_R(D, net, 16)
    costly = {R: 0.004 * R for R in range(17)}
    assert NR.best_by_total(costly, D, net)[0] < NM.best_R(D, net, 16)
