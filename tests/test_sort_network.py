"""The compare-exchange network of the FP32 move-by-move weight kernel (k_steps_weights in
csrc/steps.cu), replayed on the CPU with numpy: 8192 keys, eight per thread of 1024 in registers
(thread t holds elements 8t..8t+7); partners at distance j >= 256 are exchanged through shared
memory, 8 <= j < 256 by warp shuffle (thread t ^ j/8), j < 8 inside the thread. Each tier applies
the same rule -- the element keeps the minimum iff its bit k is clear exactly when its bit j is
clear -- which is the bitonic network, so the keys come out ascending. This pins the index
arithmetic the kernel's three tiers use; the GPU parity tests pin the weights it produces."""
import numpy as np

N, T = 8192, 1024


def network(keys):
    v = keys.reshape(T, 8).copy()          # v[t, r] = element 8t + r
    e = np.arange(N).reshape(T, 8)
    k = 2
    while k <= N:
        j = k >> 1
        while j >= 8:
            if j >= 256:                       # through shared memory: partner element e ^ j
                w = v.reshape(-1)[e ^ j]
            else:                              # warp shuffle: lane t ^ (j / 8), same register
                w = v[np.arange(T) ^ (j >> 3), :]
            keep_min = ((e & k) == 0) == ((e & j) == 0)
            v = np.where(keep_min, np.minimum(v, w), np.maximum(v, w))
            j >>= 1
        for J in (4, 2, 1):                    # inside the thread: register r against r ^ J
            if J < k:
                r = np.array([x for x in range(8) if (x ^ J) > x])
                a, b = v[:, r], v[:, r ^ J]
                asc = ((e[:, r] & k) == 0)
                lo, hi = np.minimum(a, b), np.maximum(a, b)
                v[:, r] = np.where(asc, lo, hi)
                v[:, r ^ J] = np.where(asc, hi, lo)
        k <<= 1
    return v.reshape(-1)


def test_network_sorts_with_padding_and_ties():
    rng = np.random.default_rng(7)
    for n in (1, 2, 7, 2187, 6561, 7776, 8192):
        keys = np.full(N, np.iinfo(np.uint64).max, dtype=np.uint64)   # padding: all ones
        # f bit patterns with the suffix index in the low 13 bits, as the kernel builds them;
        # a few equal f to exercise ties
        f = rng.integers(1 << 52, 1 << 62, n, dtype=np.uint64) & ~np.uint64(0x1FFF)
        if n > 4:
            f[1:4] = f[0]
        keys[:n] = f | np.arange(n, dtype=np.uint64)
        out = network(keys)
        assert np.array_equal(out, np.sort(keys)), n
        assert np.array_equal(np.sort(out[:n] & np.uint64(0x1FFF)), np.arange(n, dtype=np.uint64))
