"""A second, vectorised Philox4x32-10 in numpy, written independently of the
C oracle from the published description (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): per round, the 32x32
-> 64-bit products of counter words 0 and 2 with the two round multipliers;
the new words are (hi(w2*M1) ^ w1 ^ k0, lo(w2*M1), hi(w0*M0) ^ w3 ^ k1,
lo(w0*M0)); the key advances by the Weyl constants (golden ratio and sqrt(3)-1
in 32-bit fixed point) between rounds. Used only to generate many draws for
statistical tests and as an independent implementation to compare with."""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox(c0, c1, c2, c3, k0, k1, rounds=10):
    c = [np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3)]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = c[0] * M0
        p1 = c[2] * M1
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ np.uint64(k0)) & MASK,
             p1 & MASK,
             ((p0 >> np.uint64(32)) ^ c[3] ^ np.uint64(k1)) & MASK,
             p0 & MASK]
    return [x.astype(np.uint32) for x in c]


def uniforms(seed, rep, step, nodes):
    """u(seed, rep, step, node) for an array of nodes: word rep % 4 of
    Philox(counter=(node, step, rep//4, 0), key=(seed_lo, seed_hi)), top 24 bits."""
    nodes = np.asarray(nodes, dtype=np.uint64)
    w = philox(nodes, np.full_like(nodes, step), np.full_like(nodes, rep >> 2),
               np.zeros_like(nodes), seed & 0xFFFFFFFF, seed >> 32)[rep & 3]
    return (w >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
