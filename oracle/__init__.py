"""CPU oracle for the Pohlig-Hellman exponentiation-cipher generator.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product (``paper_1411_2484_gb300``) never imports it and never falls back to
it.  It shares no code with the CUDA library.

The arithmetic lives in ``phprng_oracle.c`` (plain C: exact integer products,
``%``, repeated squaring, one C double division for Eq. 9d).  This module
compiles it with gcc on first use and wraps it with ctypes/numpy.

Functions and the passages they follow (Beale, arXiv:1411.2484):
  mulmod, powmod ........ Introduction (definition of mod, repeated squaring)
  real .................. Eq. 9d
  generate .............. Eq. 9a-9e
  skip_stepping ......... Eq. 7 (sum formed by stepping)
  prefix_table, state_at  Eq. 7 with a coarse prefix table of the skip cycle
  dlog .................. Shanks baby-step giant-step (places s0 on the cycle)
  stats, corr ........... fused-statistics definitions of this library
  generate_many ......... threaded harness over independent instances
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phprng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None   # default Oracle instance

u64 = ctypes.c_uint64
P64 = ctypes.POINTER(ctypes.c_uint64)
PD = ctypes.POINTER(ctypes.c_double)
P32 = ctypes.POINTER(ctypes.c_uint32)


def build(force=False, src=_SRC, out=_LIB):
    """Compile phprng_oracle.c into liboracle.so (gcc -O2, no fast-math)."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall",
                           "-o", tmp, src, "-lpthread"])
    os.replace(tmp, out)
    return out


def _p64(a):
    return a.ctypes.data_as(P64)


class Oracle:
    """The oracle's functions bound to one compiled copy of phprng_oracle.c."""

    def __init__(self, so_path):
        lib = ctypes.CDLL(so_path)
        lib.or_mulmod.restype = u64
        lib.or_mulmod.argtypes = [u64, u64, u64]
        lib.or_powmod.restype = u64
        lib.or_powmod.argtypes = [u64, u64, u64]
        lib.or_real.restype = ctypes.c_double
        lib.or_real.argtypes = [u64, u64]
        lib.or_generate.restype = None
        lib.or_generate.argtypes = [u64, u64, u64, u64, P64, u64, P64, PD]
        lib.or_skip_stepping.restype = None
        lib.or_skip_stepping.argtypes = [u64, u64, u64, P64, u64]
        lib.or_prefix_table.restype = None
        lib.or_prefix_table.argtypes = [u64, u64, u64, P64, u64]
        lib.or_pref.restype = u64
        lib.or_pref.argtypes = [u64, u64, P64, u64, u64]
        lib.or_state_at.restype = None
        lib.or_state_at.argtypes = [u64, u64, u64, u64, u64, u64, P64, u64, P64]
        lib.or_dlog_many.restype = ctypes.c_int
        lib.or_dlog_many.argtypes = [u64, u64, P64, u64, P64]
        lib.or_stats.restype = None
        lib.or_stats.argtypes = [P64, u64, u64, P64, P32, PD]
        lib.or_corr.restype = None
        lib.or_corr.argtypes = [P64, P64, u64, u64, u64, P64, PD]
        lib.or_serial_hist.restype = None
        lib.or_serial_hist.argtypes = [P64, u64, u64, ctypes.c_int, u64, P64]
        lib.or_interstream_serial_hist.restype = None
        lib.or_interstream_serial_hist.argtypes = [P64, P64, u64, u64, ctypes.c_int, u64, P64]
        lib.or_poker_hist.restype = None
        lib.or_poker_hist.argtypes = [P64, u64, u64, P64]
        lib.or_runs_hist.restype = None
        lib.or_runs_hist.argtypes = [P64, u64, u64, ctypes.c_int, P64]
        lib.or_pattern_hist.restype = None
        lib.or_pattern_hist.argtypes = [u64, u64, u64, u64, u64, u64, ctypes.c_int, u64, P64]
        lib.or_pattern_const_hist.restype = None
        lib.or_pattern_const_hist.argtypes = [u64, u64, u64, u64, u64, ctypes.c_int, u64, P64]
        lib.or_pattern_region_hist.restype = None
        lib.or_pattern_region_hist.argtypes = [u64, u64, u64, u64, u64, u64, ctypes.c_int, u64, u64, P64]
        lib.or_pattern_const_region_hist.restype = None
        lib.or_pattern_const_region_hist.argtypes = [u64, u64, u64, u64, u64, ctypes.c_int, u64, u64, P64]
        lib.or_collision_hist.restype = None
        lib.or_collision_hist.argtypes = [P64, u64, u64, u64, u64, u64, P64]
        lib.or_generate_many.restype = u64
        lib.or_generate_many.argtypes = [P64, u64, u64, ctypes.c_int, P64, PD, P64]
        self.lib = lib

    def mulmod(self, x, y, n):
        return int(self.lib.or_mulmod(x, y, n))

    def powmod(self, b, e, n):
        return int(self.lib.or_powmod(b, e, n))

    def real(self, c, n):
        return float(self.lib.or_real(c, n))

    def generate(self, n, e, p, a, m, s, count):
        """Eq. 9 applied `count` times from state (m, s).

        Returns (c: uint64[count], R: float64[count], (m', s'))."""
        st = np.array([m, s], dtype=np.uint64)
        c = np.empty(count, dtype=np.uint64)
        r = np.empty(count, dtype=np.float64)
        self.lib.or_generate(n, e, p, a, _p64(st), count, _p64(c), r.ctypes.data_as(PD))
        return c, r, (int(st[0]), int(st[1]))

    def skip_stepping(self, n, p, a, m, s, k):
        """Eq. 7 from state (m, s), advancing k steps (sum formed by stepping)."""
        st = np.array([m, s], dtype=np.uint64)
        self.lib.or_skip_stepping(n, p, a, _p64(st), k)
        return int(st[0]), int(st[1])

    def PrefixTable(self, p, a, stride):
        return PrefixTable(p, a, stride, self)

    def dlog(self, p, a, s_values):
        """Discrete logs base a mod p of each s (baby-step giant-step)."""
        s = np.ascontiguousarray(np.asarray(s_values, dtype=np.uint64).reshape(-1))
        L = np.empty_like(s)
        if self.lib.or_dlog_many(p, a, _p64(s), s.size, _p64(L)) != 0:
            raise MemoryError("or_dlog_many failed")
        return L

    def stats(self, c, n):
        """(X, Y, hist[256], mean, var) of one stream's ciphertexts."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        xy = np.zeros(4, dtype=np.uint64)
        hist = np.zeros(256, dtype=np.uint32)
        mv = np.zeros(2, dtype=np.float64)
        self.lib.or_stats(_p64(c), c.size, n, _p64(xy), hist.ctypes.data_as(P32),
                          mv.ctypes.data_as(PD))
        X = int(xy[0]) | (int(xy[1]) << 64)
        Y = int(xy[2]) | (int(xy[3]) << 64)
        return X, Y, hist, float(mv[0]), float(mv[1])

    def corr(self, ca, cb, na, nb):
        """(Z, corr) for two streams' ciphertexts of equal length."""
        ca = np.ascontiguousarray(ca, dtype=np.uint64)
        cb = np.ascontiguousarray(cb, dtype=np.uint64)
        assert ca.size == cb.size
        z = np.zeros(2, dtype=np.uint64)
        out = np.zeros(1, dtype=np.float64)
        self.lib.or_corr(_p64(ca), _p64(cb), ca.size, na, nb, _p64(z),
                         out.ctypes.data_as(PD))
        return int(z[0]) | (int(z[1]) << 64), float(out[0])

    def serial_hist(self, c, n, D, B, hist=None):
        """Adds one stream's non-overlapping D-tuples (B bins per dimension)
        to hist (uint64[B**D], created when None) and returns it."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        if hist is None:
            hist = np.zeros(B ** D, dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == B ** D and hist.flags.c_contiguous
        self.lib.or_serial_hist(_p64(c), c.size, int(n), int(D), int(B), _p64(hist))
        return hist

    def interstream_serial_hist(self, c, nmod, D, B, hist=None):
        """Adds the D-tuples of the streams' numbers in interleaved order (c:
        uint64[Np, L] instance-major, nmod: the Np moduli) to hist."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        nmod = np.ascontiguousarray(nmod, dtype=np.uint64)
        Np, L = c.shape
        assert nmod.size == Np
        if hist is None:
            hist = np.zeros(B ** D, dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == B ** D and hist.flags.c_contiguous
        self.lib.or_interstream_serial_hist(_p64(c), _p64(nmod), Np, L, int(D), int(B), _p64(hist))
        return hist

    def pattern_region_hist(self, n, e, p, a, c_lo, L0, D, nb, L1, hist=None):
        """Full-period pattern of (n, e, p, a) for c0 in [c_lo, c_lo+L0), successors
        binned by floor(c / L1) and counted only inside [0, nb L1)^(D-1)."""
        if hist is None:
            hist = np.zeros(nb ** (D - 1), dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == nb ** (D - 1)
        self.lib.or_pattern_region_hist(n, e, p, a, c_lo, L0, D, nb, L1, _p64(hist))
        return hist

    def pattern_const_region_hist(self, n, e, b, c_lo, L0, D, nb, L1, hist=None):
        """The same for the constant-skip generator (skip b; b = 1 is the unit skip)."""
        if hist is None:
            hist = np.zeros(nb ** (D - 1), dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == nb ** (D - 1)
        self.lib.or_pattern_const_region_hist(n, e, b, c_lo, L0, D, nb, L1, _p64(hist))
        return hist

    def poker_hist(self, c, n, hist=None):
        """Adds one stream's five-card hands (categories 0..6) to hist (uint64[7])."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        if hist is None:
            hist = np.zeros(7, dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == 7 and hist.flags.c_contiguous
        self.lib.or_poker_hist(_p64(c), c.size, int(n), _p64(hist))
        return hist

    def runs_hist(self, c, n, lmax, hist=None):
        """Adds one stream's completed runs (bit-major, lengths capped at
        lmax) to hist (uint64[2 lmax])."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        if hist is None:
            hist = np.zeros(2 * lmax, dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == 2 * lmax and hist.flags.c_contiguous
        self.lib.or_runs_hist(_p64(c), c.size, int(n), int(lmax), _p64(hist))
        return hist

    def pattern_hist(self, n, e, p, a, c_lo, L0, D, nb, hist=None):
        """Full-period pattern of the D-tuples starting at c0 in [c_lo, c_lo+L0)
        (the O(p L0) enumeration), added to hist (uint64[nb**(D-1)])."""
        if hist is None:
            hist = np.zeros(nb ** (D - 1), dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == nb ** (D - 1) and hist.flags.c_contiguous
        self.lib.or_pattern_hist(int(n), int(e), int(p), int(a), int(c_lo), int(L0), int(D), int(nb),
                                 _p64(hist))
        return hist

    def pattern_const_hist(self, n, e, b, c_lo, L0, D, nb, hist=None):
        """Full-period pattern of the constant-skip generator (skip b; b = 1 is
        the unit skip), added to hist (uint64[nb**(D-1)])."""
        if hist is None:
            hist = np.zeros(nb ** (D - 1), dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == nb ** (D - 1) and hist.flags.c_contiguous
        self.lib.or_pattern_const_hist(int(n), int(e), int(b), int(c_lo), int(L0), int(D), int(nb),
                                       _p64(hist))
        return hist

    def collision_hist(self, c, n, S, B, H, hist=None):
        """Adds one stream's per-segment collision counts (segments of S numbers
        into B bins, counts capped at H-1) to hist (uint64[H])."""
        c = np.ascontiguousarray(c, dtype=np.uint64)
        if hist is None:
            hist = np.zeros(H, dtype=np.uint64)
        assert hist.dtype == np.uint64 and hist.size == H and hist.flags.c_contiguous
        self.lib.or_collision_hist(_p64(c), c.size, int(n), int(S), int(B), int(H), _p64(hist))
        return hist

    def generate_many(self, params, per_inst, threads=1, want_c=True, want_r=True):
        """Eq. 9 for many independent instances on `threads` threads.

        params: uint64[count, 6] rows (n, e, p, a, m, s).
        Returns (c or None, R or None, state uint64[count, 2], sink)."""
        params = np.ascontiguousarray(params, dtype=np.uint64)
        count = params.shape[0]
        c = np.empty((count, per_inst), dtype=np.uint64) if want_c else None
        r = np.empty((count, per_inst), dtype=np.float64) if want_r else None
        st = np.empty((count, 2), dtype=np.uint64)
        sink = self.lib.or_generate_many(
            _p64(params), count, per_inst, int(threads),
            _p64(c) if c is not None else None,
            r.ctypes.data_as(PD) if r is not None else None, _p64(st))
        return c, r, st, int(sink)


class PrefixTable:
    """Coarse prefix table of the skip cycle of (p, a) at a given stride."""

    def __init__(self, p, a, stride, orc=None):
        self.o = orc or _default()
        self.p, self.a, self.stride = int(p), int(a), int(stride)
        nent = (self.p - 1) // self.stride + 1
        self.table = np.zeros(nent, dtype=np.uint64)
        self.o.lib.or_prefix_table(self.p, self.a, self.stride, _p64(self.table), nent)

    def pref(self, t):
        return int(self.o.lib.or_pref(self.p, self.a, _p64(self.table), self.stride, t))

    def state_at(self, n, m0, L0, t):
        """State (m_t, s_t) after t steps from seed (m0, s0 = a^L0), Eq. 7."""
        st = np.zeros(2, dtype=np.uint64)
        self.o.lib.or_state_at(n, self.p, self.a, m0, L0, t, _p64(self.table),
                               self.stride, _p64(st))
        return int(st[0]), int(st[1])


def _default():
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def mulmod(x, y, n):
    return _default().mulmod(x, y, n)


def powmod(b, e, n):
    return _default().powmod(b, e, n)


def real(c, n):
    return _default().real(c, n)


def generate(n, e, p, a, m, s, count):
    return _default().generate(n, e, p, a, m, s, count)


def skip_stepping(n, p, a, m, s, k):
    return _default().skip_stepping(n, p, a, m, s, k)


def dlog(p, a, s_values):
    return _default().dlog(p, a, s_values)


def stats(c, n):
    return _default().stats(c, n)


def corr(ca, cb, na, nb):
    return _default().corr(ca, cb, na, nb)


def generate_many(params, per_inst, threads=1, want_c=True, want_r=True):
    return _default().generate_many(params, per_inst, threads, want_c, want_r)


def serial_hist(c, n, D, B, hist=None):
    return _default().serial_hist(c, n, D, B, hist)


def interstream_serial_hist(c, nmod, D, B, hist=None):
    return _default().interstream_serial_hist(c, nmod, D, B, hist)


def poker_hist(c, n, hist=None):
    return _default().poker_hist(c, n, hist)


def runs_hist(c, n, lmax, hist=None):
    return _default().runs_hist(c, n, lmax, hist)


def pattern_hist(n, e, p, a, c_lo, L0, D, nb, hist=None):
    return _default().pattern_hist(n, e, p, a, c_lo, L0, D, nb, hist)


def collision_hist(c, n, S, B, H, hist=None):
    return _default().collision_hist(c, n, S, B, H, hist)


# ---- Fourier test (Tests section) -------------------------------------------
# numpy's FFT serves as the library primitive of this step; everything else is
# the paper's definition written out.

def fourier_coefficients(R, M):
    """Fourier test coefficients of one stream's numbers R (in order): for each
    consecutive sequence of M numbers (a remainder left out), with x_j = R_j -
    1/2, xhat_k = M^(-1/2) sum_j x_j exp(+2 pi i j k / M) for k = 0 .. M/2-1.
    Returns complex128[sequences, M/2]."""
    R = np.asarray(R, dtype=np.float64)
    seqs = R.size // M
    x = R[: seqs * M].reshape(seqs, M) - 0.5
    # sum_j x_j exp(+2 pi i j k / M) = M * ifft(x)_k
    X = np.fft.ifft(x, axis=1) * M
    return X[:, : M // 2] / np.sqrt(M)


def fourier_bin(v, nbins, w):
    """Histogram bin of a real or imaginary part v: floor((v + w) (nbins / 2w)),
    clamped to the first and last bins outside [-w, w) (the two roundings --
    the sum, then the product with the constant nbins / 2w -- are the ones the
    library takes, so equal coefficients fall in equal bins)."""
    b = np.floor((np.asarray(v, dtype=np.float64) + w) * (nbins / (2.0 * w)))
    return np.clip(b, 0, nbins - 1).astype(np.int64)


def fourier_hist(coefs, nbins, w, hist=None):
    """Adds the real and imaginary parts of every coefficient to hist."""
    if hist is None:
        hist = np.zeros(nbins, dtype=np.uint64)
    c = np.asarray(coefs).reshape(-1)
    for part in (c.real, c.imag):
        hist += np.bincount(fourier_bin(part, nbins, w), minlength=nbins).astype(np.uint64)
    return hist


def pattern_region_hist(n, e, p, a, c_lo, L0, D, nb, L1, hist=None):
    return _default().pattern_region_hist(n, e, p, a, c_lo, L0, D, nb, L1, hist)


def pattern_const_region_hist(n, e, b, c_lo, L0, D, nb, L1, hist=None):
    return _default().pattern_const_region_hist(n, e, b, c_lo, L0, D, nb, L1, hist)


def pattern_const_hist(n, e, b, c_lo, L0, D, nb, hist=None):
    return _default().pattern_const_hist(n, e, b, c_lo, L0, D, nb, hist)
