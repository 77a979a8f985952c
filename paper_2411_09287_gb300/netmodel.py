"""Communication cost of Pi_MultVerify^R under the paper's simulated networks, and the R that
minimises it.

The paper's benchmark setting (implementation and benchmarks section) simulates three
networks: LAN (RTT 0.2 ms, 1 Gbps), MAN (RTT 12 ms, 100 Mbps) and WAN (RTT 80 ms, 40 Mbps). Its
multiplication benchmark weighs the number R of Pi_Reduce rounds: more rounds shrink the final
Pi_InnerVerify but add round trips, so slower links and larger batches want a larger R.  One GPU
has no network, so this module prices the protocol's messages instead.

Messages of Pi_MultVerify^R on D triples, as the library and the oracle send them (GR elements
of 512 bytes, hashes of 32 bytes):
  - Pi_Tran reveals the challenge r with Pi_Rec: 3 elements and 3 hashes (1632 bytes).
  - Each Pi_Reduce round sends three messages for each of h(0) and h(2): P0's [Gamma]_2, then
    P1's and P2's [m]_j. It then reveals zeta' with Pi_Rec: 9 elements and 3 hashes in all
    (4704 bytes).
  - Pi_InnerVerify on the D_R remaining pairs (D_R = D halved R times, odd lengths rounded up)
    multiplies by alpha: 3 D_R elements. The claim's product is 3 elements, and the reveal of
    Delta is 3 elements and 3 hashes.
So bytes(D, R) = 4800 + 4704 R + 1536 D_R, in 18 + 12 R messages.

Latency counts the dependent steps, each one one-way delay (RTT / 2). Messages in one step
travel at the same time on separate links.
  - Steps: 1 (reveal r) + 3 per round ([Gamma]_2, the P1/P2 exchange, the reveal of zeta')
    + 3 (Gamma of both final products, their exchange, the reveal of Delta).
  - A step lasts as long as its busiest link: bytes / bandwidth.
"""
from __future__ import annotations

from dataclasses import dataclass

GR_BYTES = 512          # one GR(2^64, 64) element
HASH_BYTES = 32
REC_BYTES = 3 * GR_BYTES + 3 * HASH_BYTES       # Pi_Rec of one element


@dataclass(frozen=True)
class Network:
    rtt_s: float        # round-trip time, seconds
    bytes_per_s: float  # link bandwidth


NETWORKS = {
    "LAN": Network(0.2e-3, 1e9 / 8),
    "MAN": Network(12e-3, 100e6 / 8),
    "WAN": Network(80e-3, 40e6 / 8),
}


def dim_after(D: int, R: int) -> int:
    """Length after R Pi_Reduce rounds (an odd length is padded with one pair)."""
    for _ in range(R):
        D = (D + 1) // 2
    return D


def verify_bytes(D: int, R: int) -> int:
    """Bytes all parties send in Pi_MultVerify^R on D triples."""
    return 2 * REC_BYTES + 3 * GR_BYTES + R * (6 * GR_BYTES + REC_BYTES) + 3 * GR_BYTES * dim_after(D, R)


def verify_messages(R: int) -> int:
    return 18 + 12 * R


def verify_steps(R: int) -> list:
    """The dependent steps of Pi_MultVerify^R, each the bytes of its busiest link."""
    rec = GR_BYTES + HASH_BYTES                      # a Pi_Rec link: one element, at most a hash
    steps = [rec]                                    # reveal r
    for _ in range(R):
        steps += [2 * GR_BYTES, 2 * GR_BYTES, rec]   # [Gamma]_2 of h(0), h(2); exchange; reveal
    return steps


def verify_time(D: int, R: int, net: Network) -> float:
    """Seconds of communication of Pi_MultVerify^R on D triples over `net`."""
    DR = dim_after(D, R)
    steps = verify_steps(R) + [GR_BYTES * (DR + 1), GR_BYTES * (DR + 1), GR_BYTES + HASH_BYTES]
    return sum(net.rtt_s / 2 + b / net.bytes_per_s for b in steps)


def best_R(D: int, net: Network, R_max: int = 24) -> int:
    """The R in [0, R_max] with the least communication time (ties: the smaller R)."""
    times = [verify_time(D, R, net) for R in range(R_max + 1)]
    return min(range(R_max + 1), key=lambda R: (times[R], R))
