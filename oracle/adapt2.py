"""The 2-byte adaptive polar encoding of JUQCS-A (Sec. 4.1), step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.1: an amplitude z = r e^{i theta} is stored as two signed bytes.
  * b1 in [-128, 128) encodes the angle: theta = pi * b1 / 128.
  * b0 in [-128, 128) encodes the magnitude: b0 = -128 means r = 0,
    b0 = 127 means r = 1, and -127 <= b0 <= 126 means
    r = (b0 + 127) (r1 - r0) / 253 + r0,
    where r0 and r1 are the minimum and maximum of |z| over the amplitudes
    with 0 < |z| < 1 in the whole state vector; they are re-tuned as the
    circuit runs.

Readings where the section is silent (each listed in the design notes):
  * rounding is round-half-to-even (numpy.rint), in FP64 here;
  * theta = atan2(Im z, Re z) in (-pi, pi]; the code 128 (theta = +pi) wraps
    to -128;
  * "r = 0" means z == 0 exactly; "r = 1" means |z| >= 1;
  * when r1 == r0 every amplitude with 0 < |z| < 1 gets b0 = -127 (r = r0);
    when no amplitude has 0 < |z| < 1, r0 = r1 = 0;
  * r0 and r1 are re-tuned after every arithmetic gate from the post-gate
    values of the whole state (decode -> exact gate -> retune -> encode);
  * permutations (X, CNOT, TOFFOLI, modular multiplication) move codes
    unchanged, and phase factors e^{i pi m/128} add m to b1 (mod 256);
    diagonal and anti-diagonal unitaries leave every |z| unchanged, so they
    keep r0, r1 (re-tuning from decoded values would only move r1 by an
    ulp of rounding);
  * the encoding does not renormalise.

Word layout shared with the device state: one little-endian 16-bit word per
amplitude, low byte b0, high byte b1 (two's complement).
"""
import math
import numpy as np

from . import statevec as sv

PI = math.pi


def retune(z):
    """(r0, r1) = (min, max) of |z| over the entries with 0 < |z| < 1."""
    m = np.abs(z)
    sel = m[(m > 0.0) & (m < 1.0)]
    if sel.size == 0:
        return 0.0, 0.0
    return float(sel.min()), float(sel.max())


def encode_real(z, r0, r1):
    """Pre-rounding code values (q0, q1): q0 = (|z| - r0) * 253 / (r1 - r0)
    (code b0 = rint(q0) - 127), q1 = theta * 128 / pi (code b1 = rint(q1))."""
    z = np.asarray(z, dtype=np.complex128)
    m = np.abs(z)
    if r1 > r0:
        q0 = (m - r0) * 253.0 / (r1 - r0)
    else:
        q0 = np.zeros(m.shape)
    q1 = np.arctan2(z.imag, z.real) * 128.0 / PI
    return q0, q1


def encode(z, r0, r1):
    """Encode complex128 values with parameters (r0, r1) into (b0, b1) int8."""
    z = np.asarray(z, dtype=np.complex128)
    m = np.abs(z)
    q0, q1 = encode_real(z, r0, r1)
    b0 = np.clip(np.rint(q0) - 127.0, -127.0, 126.0)
    b0 = np.where(m >= 1.0, 127.0, b0)
    b0 = np.where(z == 0, -128.0, b0)
    b1 = np.rint(q1)
    b1 = np.where(b1 >= 128.0, b1 - 256.0, b1)
    b1 = np.where(z == 0, 0.0, b1)
    return b0.astype(np.int8), b1.astype(np.int8)


def _angle_table():
    """(cos, sin) of theta = pi b1 / 128 for b1 = -128..127 (index b1 + 128).

    The values for 0 <= b1 < 64 are computed directly; the others follow by
    exact quarter turns, (c, s) -> (-s, c), so that two amplitudes of equal
    magnitude code and angles pi apart cancel exactly, as they do in exact
    arithmetic."""
    k = np.arange(64)
    c = np.cos(PI * k / 128.0)
    sn = np.sin(PI * k / 128.0)
    cs = np.empty(256)
    ss = np.empty(256)
    for quarter in range(4):           # b1 = k + 64 * quarter - 128
        idx = k + 64 * quarter
        rc, rs = c, sn
        for _ in range((quarter + 2) % 4):   # rotate by (quarter - 2) quarter turns
            rc, rs = -rs, rc
        cs[idx] = rc
        ss[idx] = rs
    return cs, ss


ANGLE_COS, ANGLE_SIN = _angle_table()


def decode(b0, b1, r0, r1):
    """Decode (b0, b1) codes with parameters (r0, r1) into complex128."""
    b0 = np.asarray(b0, dtype=np.int64)
    b1 = np.asarray(b1, dtype=np.int64)
    r = (b0 + 127) * (r1 - r0) / 253.0 + r0
    r = np.where(b0 == -128, 0.0, r)
    r = np.where(b0 == 127, 1.0, r)
    return r * ANGLE_COS[b1 + 128] + 1j * (r * ANGLE_SIN[b1 + 128])


def pack(b0, b1):
    """Codes -> uint16 words (low byte b0, high byte b1)."""
    return (np.asarray(b0, np.int8).view(np.uint8).astype(np.uint16)
            | (np.asarray(b1, np.int8).view(np.uint8).astype(np.uint16) << 8))


def unpack(words):
    w = np.asarray(words).view(np.uint16)
    b0 = (w & 0xFF).astype(np.uint8).view(np.int8)
    b1 = (w >> 8).astype(np.uint8).view(np.int8)
    return b0, b1


class AState:
    """An N-qubit state held as codes (b0, b1) plus the global (r0, r1)."""

    def __init__(self, N, b0, b1, r0, r1):
        self.N, self.b0, self.b1, self.r0, self.r1 = N, b0, b1, float(r0), float(r1)

    @classmethod
    def zero(cls, N):
        """|0..0>: a(0) = 1 -> b0 = 127 (r = 1), all others b0 = -128 (r = 0);
        no amplitude has 0 < |z| < 1, so r0 = r1 = 0."""
        b0 = np.full(1 << N, -128, dtype=np.int8)
        b1 = np.zeros(1 << N, dtype=np.int8)
        b0[0] = 127
        return cls(N, b0, b1, 0.0, 0.0)

    @classmethod
    def from_complex(cls, N, z):
        r0, r1 = retune(z)
        b0, b1 = encode(z, r0, r1)
        return cls(N, b0, b1, r0, r1)

    def copy(self):
        return AState(self.N, self.b0.copy(), self.b1.copy(), self.r0, self.r1)

    def to_complex(self):
        return decode(self.b0, self.b1, self.r0, self.r1)

    def words(self):
        return pack(self.b0, self.b1)

    # --- arithmetic gate: decode -> exact FP64 gate -> retune -> encode -----
    def arithmetic(self, fn, retune_range=True):
        z = self.to_complex()
        fn(z)
        if retune_range:
            self.r0, self.r1 = retune(z)
        self.b0, self.b1 = encode(z, self.r0, self.r1)
        return self

    # --- code-only operations ------------------------------------------------
    def permute(self, fn_index):
        """Apply an index permutation given as a function mapping a
        complex128 vector in place; codes move with their amplitudes."""
        idx = np.arange(1 << self.N, dtype=np.float64).astype(np.complex128)
        fn_index(idx)
        src = idx.real.astype(np.int64)
        self.b0 = self.b0[src]
        self.b1 = self.b1[src]
        return self

    def phase_steps(self, steps):
        """Multiply amplitude i by e^{i pi steps[i]/128}: b1 += steps (mod 256)
        for every amplitude with r != 0."""
        s = np.asarray(steps, dtype=np.int64)
        nb = ((self.b1.astype(np.int64) + s + 128) % 256) - 128
        nb = np.where(self.b0 == -128, self.b1.astype(np.int64), nb)
        self.b1 = nb.astype(np.int8)
        return self
