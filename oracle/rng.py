"""Disorder potential of the Anderson model (oracle side).

The paper draws the on-site energies eps_{i;j;k} from the box distribution
on [-w/2, w/2] (Section 3, the paragraph following Eq. (1)); it does not say
which random number generator produced them.  Reading used throughout this
project: eps at lattice site ``idx`` is

    u   = (SplitMix64_idx(seed) >> 11) * 2**-53          in [0, 1)
    eps = W * (u - 1/2)                                  in [-W/2, W/2)

where SplitMix64_idx(seed) is the idx-th output (idx = 0, 1, ...) of
Steele, Lea & Flood's SplitMix64 generator seeded with ``seed``: the state
advances by the golden-ratio increment 0x9E3779B97F4A7C15 and each state is
passed through the variant-13 finaliser (shift 30, multiply 0xBF58476D1CE4E5B9,
shift 27, multiply 0x94D049BB133111EB, shift 31).  Because the idx-th state
is seed + (idx+1) * increment, each output is computed independently of the
others (a counter-based generator).

This file is the oracle's own implementation of that published definition;
the GPU library implements the same definition separately.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, offset=0):
    """Outputs offset .. offset+count-1 of SplitMix64 seeded with ``seed``.

    Returns a uint64 array.  Arithmetic is modulo 2**64 (numpy uint64 wraps).
    """
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, offset=0):
    """u_idx = top 53 bits of the idx-th SplitMix64 output, times 2**-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def potential(L, W, seed):
    """On-site energies eps[idx], idx = x + L*(y + L*z), box distribution
    on [-W/2, W/2) (Section 3, after Eq. (1)).  FP64, length L**3."""
    n = int(L) ** 3
    u = uniform01(seed, n)
    return np.float64(W) * (u - 0.5)


def hoppings(L, seed, width=1.0):
    """Random hopping amplitudes of the off-diagonal Anderson model (Section
    7, Table 6: the randomness moved from the diagonal to the off-diagonal
    entries, uniform on [-1/2, 1/2] for width 1).  Reading: the bond from
    site s to its +x, +y, +z neighbour (d = 0, 1, 2) gets
    t[s, d] = width * (u_{3s+d} - 1/2), u the same SplitMix64 stream as
    `potential`, indexed 3s + d.  FP64, shape (L**3, 3)."""
    n = int(L) ** 3
    u = uniform01(seed, 3 * n)
    return (np.float64(width) * (u - 0.5)).reshape(n, 3)
