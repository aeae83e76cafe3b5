"""cuRAND's host-side Philox4_32_10 generator as an external reference for
Philox4x32-10 (Salmon et al., SC'11), test infrastructure only.

The generator runs on the CPU (no GPU needed).  In its default ordering,
output block b (four 32-bit words) is the Philox4x32-10 block of counter
(lo32(b >> 16), hi32(b >> 16), b & 0xFFFF, 0) under the key (lo32(seed),
hi32(seed)), and an offset of 4 b outputs starts the stream at block b.
That layout was established by calling the library and is what the tests
check against; counter word 3 is always 0 there.
"""
import ctypes
import ctypes.util
import os

import numpy as np

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # curandRngType_t


def _load():
    cands = [ctypes.util.find_library("curand")]
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cands += [os.path.join(home, "lib64", n) for n in ("libcurand.so", "libcurand.so.10")]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


_lib = _load()


def available():
    return _lib is not None


def blocks(seed, b0, n):
    """n consecutive output blocks starting at block b0: uint32 array (n, 4)."""
    gen = ctypes.c_void_p()
    assert _lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert _lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert _lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * b0)) == 0
        buf = (ctypes.c_uint * (4 * n))()
        assert _lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * n)) == 0
    finally:
        _lib.curandDestroyGenerator(gen)
    return np.frombuffer(buf, dtype=np.uint32).reshape(n, 4).copy()


def counters(b0, n):
    """The Philox counters of output blocks b0 .. b0 + n - 1: uint32 array (n, 4)."""
    b = np.arange(n, dtype=np.uint64) + np.uint64(b0)
    hi = b >> np.uint64(16)
    c = np.zeros((n, 4), dtype=np.uint32)
    c[:, 0] = (hi & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    c[:, 1] = (hi >> np.uint64(32)).astype(np.uint32)
    c[:, 2] = (b & np.uint64(0xFFFF)).astype(np.uint32)
    return c


# (seed, first block, blocks): counter word 2 across its 16-bit range and its
# wrap into words 0/1, word 0 near its top, word 1 non-zero, all-ones seed
CASES = [(0, 0, 4096), (0x0123456789ABCDEF, 65530, 16), (2 ** 64 - 1, (0xFFFFFFF0 << 16) + 65533, 40),
         (0xFEDCBA9876543210, ((3 << 32) + 12345) << 16 | 777, 8), (42, (0x2A5 << 48) + 3, 8)]
