"""Three simulated parties, their <.> sharings and the message ledger (oracle; test infra only).

Paper, Sec. 2 "Notation": <x> = ([r_x], m_x) with m_x = r_x + x and r_x = [r_x]_1 + [r_x]_2;
P1 holds (m_x, [r_x]_1), P2 holds (m_x, [r_x]_2), P0 holds ([r_x]_1, [r_x]_2).  The same holds for
<.>^{l[x]} over GR(2^l, d).  Linear maps with public coefficients act on every component (Sec. 2:
"linear homomorphic property").

Each party keeps its own copy of every component it holds; a message is a copy from the sender's
buffer to the receiver's, recorded in the ledger as (src, dst, phase, protocol, bytes).  A fault
site, when armed, XORs a mask into one element of one delivered message (a host-side model of a
cheating sender; nothing here touches a GPU).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .chacha import PAIR_01, PAIR_02, PAIR_12, derive_pair_keys, prf_u64
from .galois import GR, gr64

# Stream components: which pair key a stream uses.
C_R1, C_R2, C_M12, C_G1, C_TB1, C_TB2 = 1, 2, 3, 4, 5, 6
_COMP_PAIR = {C_R1: PAIR_01, C_R2: PAIR_02, C_M12: PAIR_12, C_G1: PAIR_01,
              C_TB1: PAIR_01, C_TB2: PAIR_02}

# Stream purposes (tag = purpose << 4 | component).
P_SHARE, P_MULT, P_INNER, P_TRUNC_BITS, P_TRUNC_P, P_TRUNC_Q = 0x01, 0x02, 0x03, 0x04, 0x05, 0x06
# non-linear layers (Sec. 4.3): daBits, edaBits, AND gates, their arithmetic products, the final
# product of ReLU / compare-select
P_DABIT, P_EDABIT, P_AND, P_EDA_MULT, P_EDA_INNER, P_DA_MULT1, P_DA_MULT2, P_NL_MULT = (
    0x07, 0x08, 0x09, 0x0A, 0x0B, 0x0C, 0x0D, 0x0E)
P_VER_R, P_VER_ZETA, P_VER_H0, P_VER_H2, P_VER_ALPHA, P_VER_XA, P_VER_DELTA = (
    0x10, 0x11, 0x12, 0x13, 0x14, 0x15, 0x16)

OFFLINE, ONLINE, VERIFY = "offline", "online", "verify"

FAULT_SITES = ("GAMMA2", "MZ1", "MZ2", "MX_COPY_P1", "REC_MSG", "HIGH_BIT", "TRUNC_D1")


def tag(purpose: int, comp: int) -> int:
    return (purpose << 4) | comp


def obj_id(call_id: int, batch: int = 0, sub: int = 0) -> int:
    """Object id of a PRF stream: caller's call id (< 2^44), batch (< 16) and sub index (< 2^16)."""
    assert 0 <= call_id < (1 << 44) and 0 <= batch < 16 and 0 <= sub < (1 << 16)
    return (call_id << 20) | (batch << 16) | sub


@dataclass
class Shared:
    """<x>: every party's copy of every component it holds (arrays of equal shape)."""
    p0_r1: np.ndarray
    p0_r2: np.ndarray
    p1_m: np.ndarray
    p1_r1: np.ndarray
    p2_m: np.ndarray
    p2_r2: np.ndarray

    FIELDS = ("p0_r1", "p0_r2", "p1_m", "p1_r1", "p2_m", "p2_r2")

    def map(self, fn) -> "Shared":
        return Shared(*(fn(getattr(self, f)) for f in self.FIELDS))

    def zip(self, other: "Shared", fn) -> "Shared":
        return Shared(*(fn(getattr(self, f), getattr(other, f)) for f in self.FIELDS))

    def as_tuple(self):
        return tuple(getattr(self, f) for f in self.FIELDS)

    @property
    def shape(self):
        return self.p1_m.shape

    def __getitem__(self, idx) -> "Shared":
        return self.map(lambda a: a[idx])

    def open(self, mask=np.uint64(0xFFFFFFFFFFFFFFFF)) -> np.ndarray:
        """The shared value from P1's and P2's views (no messages; for tests)."""
        v1 = (self.p1_m - self.p1_r1 - self.p2_r2) & mask
        return v1


def shared_zeros(shape, dtype=np.uint64) -> Shared:
    return Shared(*(np.zeros(shape, dtype=dtype) for _ in range(6)))


def shared_concat(parts, axis=0) -> Shared:
    return Shared(*(np.concatenate([getattr(p, f) for p in parts], axis=axis)
                    for f in Shared.FIELDS))


@dataclass
class LedgerEntry:
    src: int
    dst: int
    phase: str
    proto: str
    nbytes: int


@dataclass
class Session:
    """Keys, ledger and fault table of one three-party run."""
    seed: bytes
    gr: GR = field(default_factory=gr64)
    reduce_mode: str = "x"  # "x": third point x (default); "zeta2": points 0,1,2 at 2*zeta'
    ledger: list = field(default_factory=list)
    faults: dict = field(default_factory=dict)
    forced: dict = field(default_factory=dict)   # (purpose, obj) -> challenge value (tests)

    def __post_init__(self):
        assert len(self.seed) == 32
        self.keys = derive_pair_keys(self.seed)
        self.mask = self.gr.mask

    # ---- randomness ------------------------------------------------------------------------
    def prf(self, comp: int, purpose: int, obj: int, count: int, start: int = 0) -> np.ndarray:
        key = self.keys[_COMP_PAIR[comp]]
        return prf_u64(key, tag(purpose, comp), obj, start, count) & self.mask

    def prf_gr(self, comp: int, purpose: int, obj: int, n: int = None) -> np.ndarray:
        """GR elements from a stream: element i, coefficient c is stream word i*d + c."""
        d = self.gr.d
        if n is None:
            return self.prf(comp, purpose, obj, d)
        return self.prf(comp, purpose, obj, n * d).reshape(n, d)

    def wire(self, arr) -> np.ndarray:
        """The words a party puts on the wire for `arr` (what Pi_Rec hashes)."""
        return np.asarray(arr, dtype=np.uint64)

    # ---- messages ----------------------------------------------------------------------------
    def arm_fault(self, site: str, index: int, xor_mask: int):
        assert site in FAULT_SITES
        self.faults[site] = (int(index), int(xor_mask))

    def send(self, src: int, dst: int, phase: str, proto: str, arr, site: str = None,
             nbytes: int = None) -> np.ndarray:
        arr = np.array(arr, dtype=np.uint64, copy=True)
        if nbytes is None:
            nbytes = arr.size * 8 * self.gr.ell // 64 if self.gr.ell < 64 else arr.size * 8
        self.ledger.append(LedgerEntry(src, dst, phase, proto, nbytes))
        if site is not None and site in self.faults:
            idx, m = self.faults.pop(site)
            flat = arr.reshape(-1)
            flat[idx % max(flat.size, 1)] ^= np.uint64(m)
            arr = (flat & self.mask).reshape(arr.shape)
        return arr

    def send_hash(self, src: int, dst: int, phase: str, proto: str, digest: bytes) -> bytes:
        self.ledger.append(LedgerEntry(src, dst, phase, proto, len(digest)))
        return digest

    def ledger_bytes(self, phase=None, proto=None) -> int:
        return sum(e.nbytes for e in self.ledger
                   if (phase is None or e.phase == phase) and (proto is None or e.proto == proto))
