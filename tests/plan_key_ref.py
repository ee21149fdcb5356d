"""The documented structural key of the plan cache, written out with numpy
(every stored index adds mix(mix(tag << 56 ^ position) + value) modulo 2^64;
mix is the SplitMix64 finaliser, applied to z + 0x9E3779B97F4A7C15)."""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def mix(z):
    with np.errstate(over="ignore"):   # arithmetic modulo 2^64
        z = np.asarray(z, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def plan_key(m, n, rowptr, colidx, dtype_code):
    with np.errstate(over="ignore"):
        rp = np.asarray(rowptr, dtype=np.int32).view(np.uint32).astype(np.uint64)
        ci = np.asarray(colidx, dtype=np.int32).view(np.uint32).astype(np.uint64)
        t1 = mix(mix((np.uint64(1) << np.uint64(56)) ^ np.arange(len(rp), dtype=np.uint64)) + rp)
        t2 = mix(mix((np.uint64(2) << np.uint64(56)) ^ np.arange(len(ci), dtype=np.uint64)) + ci)
        s = np.uint64(t1.sum(dtype=np.uint64)) + np.uint64(t2.sum(dtype=np.uint64))
        nnz = len(ci)
        s = s + mix(np.uint64(4 * m)) + mix(np.uint64(4 * n + 1)) + mix(np.uint64(4 * nnz + 2)) + \
            mix(np.uint64(4 * dtype_code + 3))
        return int(mix(s))
