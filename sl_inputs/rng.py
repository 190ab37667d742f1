"""Counter-based SplitMix64 streams (vectorised over the counter)."""
import numpy as np

_G = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix64_scalar(z):
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def _mix64_inplace(z):
    t = np.right_shift(z, np.uint64(30))
    np.bitwise_xor(z, t, out=z)
    np.multiply(z, _M1, out=z)
    np.right_shift(z, np.uint64(27), out=t)
    np.bitwise_xor(z, t, out=z)
    np.multiply(z, _M2, out=z)
    np.right_shift(z, np.uint64(31), out=t)
    np.bitwise_xor(z, t, out=z)
    return z


def splitmix64(seed, stream, idx):
    """64-bit value number `idx` (array) of stream `stream` under `seed`."""
    key = _mix64_scalar((int(seed) * _G + int(stream)) & _MASK)
    z = np.array(idx, dtype=np.uint64, copy=True, ndmin=1)
    np.add(z, np.uint64(1), out=z)
    np.multiply(z, np.uint64(_G), out=z)
    np.add(z, np.uint64(key), out=z)
    z = _mix64_inplace(z)
    return z if np.ndim(idx) else z[0]


def uniform01(seed, stream, idx):
    """Uniform doubles in [0, 1) with 53 random bits."""
    z = splitmix64(seed, stream, idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal01(seed, stream, idx):
    """Standard normal draws by Box-Muller on two uniform streams."""
    u1 = uniform01(seed, stream, idx)
    u2 = uniform01(seed, stream + 1000003, idx)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
