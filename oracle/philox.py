"""Philox4x64-10 and the Gaussian sketch matrix Omega (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper draws the columns of Omega with independent standard Gaussian
entries (Section IV, Alg. 1) and notes that the method does not depend
on the quality of the generator.  To make the CPU oracle and the GPU path use
the identical Omega, both implement the same counter-based generator from its
published definition: Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).

Definition used (one round, 64-bit words, key (k0, k1)):
    (hi0, lo0) = M0 * c0      (full 128-bit product), M0 = 0xD2E7470EE14C6C93
    (hi1, lo1) = M1 * c2,                              M1 = 0xCA5A826395121157
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
and between rounds the key is bumped by the Weyl constants
    W0 = 0x9E3779B97F4A7C15, W1 = 0xBB67AE8584CAA73B.

Omega layout and counters: Omega is n x l complex, row-major; element
(r, c) uses counter (r*l + c, bond, sweep, chain) and key (seed, stream) with
stream 0 for the sketch and 1 for accuracy-check probes.  Output words w0, w1
become uniforms u = ((w >> 12) + 0.5) * 2^-52 in (0, 1) (exact in FP64), and the Box-Muller
transform gives Re = rho cos(2 pi u2), Im = rho sin(2 pi u2),
rho = sqrt(-2 ln u1): real and imaginary parts are independent N(0, 1).
"""
import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK64 = (1 << 64) - 1


def philox4x64_10(counter, key):
    """One Philox4x64-10 block on Python integers: returns four 64-bit words."""
    c0, c1, c2, c3 = (int(x) & MASK64 for x in counter)
    k0, k1 = (int(x) & MASK64 for x in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK64
            k1 = (k1 + W1) & MASK64
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0, c1, c2, c3)


def _mulhilo64(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays, via 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo, a_hi = a & m32, a >> s32
    b_lo, b_hi = b & m32, b >> s32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> s32) + (lh & m32) + (hl & m32)
    lo = (ll & m32) | ((mid & m32) << s32)
    hi = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    return hi, lo


def philox4x64_10_array(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x64-10 over uint64 arrays (same definition as above)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64).copy() for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0)
    k1 = np.uint64(k1)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + W0) & MASK64)
            k1 = np.uint64((int(k1) + W1) & MASK64)
        hi0, lo0 = _mulhilo64(np.uint64(M0), c0)
        hi1, lo1 = _mulhilo64(np.uint64(M1), c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform53(w):
    """64-bit word -> double in the open interval (0, 1)."""
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def gaussian_omega(n, l, seed, bond=0, sweep=0, chain=0, stream=0):
    """The n x l complex Gaussian sketch matrix of Alg. 1.

    Real and imaginary parts are iid N(0, 1) (the paper's "standard Gaussian",
    read per component for complex A).
    """
    if n == 0 or l == 0:
        return np.zeros((n, l), dtype=np.complex128)
    idx = np.arange(n * l, dtype=np.uint64)
    z = np.zeros_like(idx)
    w0, w1, _, _ = philox4x64_10_array(idx, z + np.uint64(bond), z + np.uint64(sweep),
                                       z + np.uint64(chain), seed & MASK64, stream & MASK64)
    u1 = uniform53(w0)
    u2 = uniform53(w1)
    rho = np.sqrt(-2.0 * np.log(u1))
    om = rho * np.cos(2.0 * np.pi * u2) + 1j * (rho * np.sin(2.0 * np.pi * u2))
    return om.reshape(n, l)
