"""cuRAND's host-side Philox4x32-10 generator, run through ctypes.

Used only as an independent implementation to pin the oracle's Philox.
The generator hands out its stream in 65,536 interleaved subsequences:
4-tuple number p (counting from offset/4) is the block function at counter
(low 32 bits of p >> 16, high 32 bits of p >> 16, p & 0xffff, 0) under the
key (seed low 32 bits, seed high 32 bits).
"""
import ctypes
import ctypes.util
import os

import numpy as np

_PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10 in curand.h


def load():
    cands = ["/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10"]
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        if os.path.exists(c) or not c.startswith("/"):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


def generate(lib, seed: int, offset_words: int, n_words: int) -> np.ndarray:
    gen = ctypes.c_void_p()
    st = lib.curandCreateGeneratorHost(ctypes.byref(gen), ctypes.c_int(_PHILOX))
    if st != 0:
        raise RuntimeError(f"curandCreateGeneratorHost: {st}")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        st = lib.curandGenerate(gen, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                                ctypes.c_size_t(n_words))
        assert st == 0, st
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def counter_of(p: int):
    q = p >> 16
    return (q & 0xFFFFFFFF, (q >> 32) & 0xFFFFFFFF, p & 0xFFFF, 0)
