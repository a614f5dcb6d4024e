"""Philox4x64-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE ONLY: this module belongs to the FP64 CPU oracle.  Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg may import it;
the CUDA path carries its own implementation and never calls this one.

Source: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (the Philox-4x64 round function, its two
multipliers and its Weyl key schedule; 10 rounds).

The randomized CP-ALS paper (Bharadwaj et al., arXiv 2210.05105) leaves the
generator open; the draws of its Algorithms 3 and 5 only need i.i.d. uniforms.
We fix one counter-based generator so that the oracle and the GPU can be given
bit-identical uniforms: counter = (j, k, n, s) for sample j, factor k, solved
mode n and sweep s; key = (seed, stream).  The uniform is the top 53 bits of
output word 0 scaled by 2^-53, so u lies in [0, 1) exactly in binary64.

Everything is vectorised over numpy uint64 arrays; 64x64->128 products are
formed from 32-bit limbs (schoolbook multiplication), which numpy evaluates
exactly in uint64 arithmetic.
"""
import numpy as np

# Philox-4x64 multipliers and Weyl increments (golden ratio, sqrt(3)-1), SC'11.
M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
ROUNDS = 10

_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a, b):
    """Exact 128-bit product of uint64 a and b, returned as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    # middle column: carries from the low word plus the two cross terms
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64(ctr, key, rounds=ROUNDS):
    """Philox4x64-R bijection.

    ctr: uint64 array of shape (4, ...) ; key: uint64 array of shape (2, ...)
    (broadcastable).  Returns a uint64 array of shape (4, ...).
    One round maps (x0, x1, x2, x3) with key (k0, k1) to
    (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0));
    between rounds the key is advanced by (W0, W1).
    """
    with np.errstate(over="ignore"):
        x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
        k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
        for r in range(rounds):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = _mulhilo64(M0, x0)
            hi1, lo1 = _mulhilo64(M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack(np.broadcast_arrays(x0, x1, x2, x3))


def uniform01(word):
    """Map a uint64 word to a binary64 in [0, 1): top 53 bits times 2^-53."""
    w = np.asarray(word, dtype=np.uint64) >> np.uint64(11)
    return w.astype(np.float64) * (2.0 ** -53)


def draw_uniforms(seed, stream, j, k, n, s):
    """Uniforms u(seed, stream; j, k, n, s) for arrays/scalars j, k, n, s."""
    j = np.asarray(j, dtype=np.uint64)
    shape = j.shape
    ctr = [j,
           np.full(shape, k, dtype=np.uint64),
           np.full(shape, n, dtype=np.uint64),
           np.full(shape, s, dtype=np.uint64)]
    key = [np.full(shape, seed, dtype=np.uint64), np.full(shape, stream, dtype=np.uint64)]
    return uniform01(philox4x64(ctr, key)[0])


# stream ids of the key's second word, one per use of randomness in the method
STREAM_ARLS = 0
STREAM_STS = 1
STREAM_INIT = 2


def gaussian_factors(dims, R, seed):
    """Unit-variance Gaussian factors of Algorithm 1's initialisation drawn from the
    same generator: entry (i, r) of U_k is the Box-Muller transform (Box and
    Muller, 1958) of two uniforms from Philox4x64-10 with key (seed, 2) and
    counter (i, r, k, 0): u1 = (top 53 bits of word 0 + 1) 2^-53 in (0, 1],
    u2 = top 53 bits of word 1 times 2^-53, z = sqrt(-2 ln u1) cos(2 pi u2)
    in binary64, rounded to float32.  Returns a list of (I_k, R) float32."""
    out = []
    for k, I in enumerate(dims):
        i = np.repeat(np.arange(int(I), dtype=np.uint64), R)
        r = np.tile(np.arange(R, dtype=np.uint64), int(I))
        ctr = [i, r, np.full(i.shape, k, dtype=np.uint64), np.zeros(i.shape, dtype=np.uint64)]
        key = [np.full(i.shape, seed, dtype=np.uint64), np.full(i.shape, STREAM_INIT, dtype=np.uint64)]
        w = philox4x64(ctr, key)
        u1 = ((w[0] >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * (2.0 ** -53)
        u2 = (w[1] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        out.append(z.astype(np.float32).reshape(int(I), R))
    return out
