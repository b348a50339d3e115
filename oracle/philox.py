"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11, section 3.2).

One round maps the counter (c0,c1,c2,c3) under key (k0,k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.

The draws the PIC step consumes are addressed by
    counter = (uid, step, call, species),  key = (seed & 0xffffffff, seed >> 32)
so a particle's random numbers depend only on its identity and the step, never
on its position in memory (the kernels keep particles in cell order, the oracle
in any order).  The null-collision test of every particle uses the cheaper
Philox2x32-10 (same paper) at counter (uid, step | species << 31) under the key
(seed & 0xffffffff) ^ (seed >> 32); the draws of actual collision candidates
come from Philox4x32-10.

Uniform conversion: u = ((x >> 9) + 0.5) * 2**-23, which lies in (0, 1) and is
exact in float32 (at most 24 significant bits).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Apply Philox4x32-R to arrays of counters; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint32).copy() for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (np.array(c, dtype=np.uint32) for c in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for r in range(rounds):
        if r > 0:
            k0 = np.uint32((int(k0) + int(W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(W1)) & 0xFFFFFFFF)
        p0 = M0 * c0.astype(np.uint64)
        p1 = M1 * c2.astype(np.uint64)
        hi0 = (p0 >> _SH).astype(np.uint32)
        lo0 = (p0 & _MASK).astype(np.uint32)
        hi1 = (p1 >> _SH).astype(np.uint32)
        lo1 = (p1 & _MASK).astype(np.uint32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


M2 = np.uint64(0xD256D193)


def philox2x32(c0, c1, k, rounds=10):
    """Philox2x32-R (same paper): round (c0, c1; k) -> (hi(M c0) ^ k ^ c1,
    lo(M c0)) with M = 0xD256D193, key bumped by 0x9E3779B9 between rounds."""
    c0 = np.array(c0, dtype=np.uint32)
    c1 = np.array(c1, dtype=np.uint32)
    c0, c1 = np.broadcast_arrays(c0, c1)
    c0, c1 = np.array(c0, dtype=np.uint32), np.array(c1, dtype=np.uint32)
    k = int(k) & 0xFFFFFFFF
    for r in range(rounds):
        if r > 0:
            k = (k + int(W0)) & 0xFFFFFFFF
        p = M2 * c0.astype(np.uint64)
        hi = (p >> _SH).astype(np.uint32)
        lo = (p & _MASK).astype(np.uint32)
        c0, c1 = hi ^ np.uint32(k) ^ c1, lo
    return c0, c1


def null_draw(uid, step, species, seed, dtype=np.float32):
    """The per-particle uniform of the null-collision test: first output of
    Philox2x32-10 at counter (uid, step | species << 31) under the key
    (seed & 0xffffffff) ^ (seed >> 32)."""
    uid = np.asarray(uid, dtype=np.uint32)
    c1 = np.uint32((step & 0x7FFFFFFF) | (species << 31))
    out, _ = philox2x32(uid, np.full(uid.shape, c1, np.uint32), (seed & 0xFFFFFFFF) ^ ((seed >> 32) & 0xFFFFFFFF))
    return to_uniform(out, dtype)


def to_uniform(x, dtype=np.float32):
    """(x >> 9) + 0.5 scaled by 2**-23: exact in float32, strictly inside (0,1)."""
    x = np.asarray(x, dtype=np.uint32)
    m = (x >> np.uint32(9)).astype(np.int64) * 2 + 1          # odd integer < 2**24
    return (m.astype(dtype) * dtype(2.0 ** -24)).astype(dtype)


def draws(uid, step, call, species, seed, dtype=np.float32):
    """Four uniforms per particle for (uid, step, call, species) under `seed`."""
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    uid = np.asarray(uid, dtype=np.uint32)
    n = uid.shape
    out = philox4x32(uid, np.full(n, step, np.uint32), np.full(n, call, np.uint32),
                     np.full(n, species, np.uint32), k0, k1)
    return tuple(to_uniform(o, dtype) for o in out)
