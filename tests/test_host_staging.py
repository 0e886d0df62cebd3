"""Index arithmetic of the class-split filter's pass 1, modelled on the host
for one CTA of T threads (T a multiple of 32 in [640, 1024]) and one
half-tile (16 columns per thread).  Each thread counts its columns per class
from the class masks of its word, the counts go to the padded cursor array
(cursor (q, t) at q*Tp + t + 4*(t // 32), Tp >= T + T/8 a multiple of 32),
thread t scans the chunk of counts 16t..16t+15 of the class-major order and
writes back exclusive positions, and the scatter moves each key to its
cursor.  (The kernel packs both half-tiles' counts into one word and scans
them together; the halves do not interact, so one is modelled.)  The model
checks what the kernel's indexing relies on: a chunk lies inside one class
and is 16 words contiguous and 16-byte aligned in the padded array, the
padded array fits its region, the positions are a permutation of the staged
entries in class order (thread order, then column order, inside a class),
the class starts written by the chunk heads equal the class offsets, the
chunk reads are free of bank conflicts, and so are a warp's cursor accesses,
whatever class each lane's column has.
"""
import numpy as np
import pytest

SMEM_WORDS = 57344            # the filter kernel's dynamic shared memory in words
STAGE = 16 * 1024             # staging entries (keys and columns each)


def cpos(q, t, T):
    Tp = (T + T // 8 + 31) // 32 * 32
    return q * Tp + t + 4 * (t // 32)


def chunk_start(t, T):
    q, t0 = (16 * t) // T, 16 * t - ((16 * t) // T) * T
    return cpos(q, t0, T)


def class_of_columns(rng, T, valid_frac=1.0):
    """Class (0..15) of each of the 16 columns of every thread's half word,
    -1 for a column past p."""
    cls = rng.integers(0, 16, size=(T, 16))
    if valid_frac < 1.0:
        cut = int(T * 16 * valid_frac)
        flat = cls.reshape(-1)
        flat[cut:] = -1                          # the ragged end of the last tile
    return cls


def run_half_tile(cls):
    T = cls.shape[0]
    Tp = (T + T // 8 + 31) // 32 * 32
    assert Tp % 32 == 0
    nwarps = T // 32
    assert 2 * STAGE + 16 * Tp <= SMEM_WORDS
    cur = np.full(16 * Tp, -1, dtype=np.int64)
    # counts (the popcounts of the class masks), at q*Tp + tt
    for t in range(T):
        tt = t + 4 * (t // 32)
        for q in range(16):
            assert q * Tp + tt == cpos(q, t, T)
            cur[q * Tp + tt] = int(np.sum(cls[t] == q))
    # chunk scan
    chunk_sum = np.zeros(T, dtype=np.int64)
    for t in range(T):
        start = chunk_start(t, T)
        q, t0 = (16 * t) // T, (16 * t) % T
        assert start % 4 == 0                                       # 16-byte aligned
        assert all(cpos(q, t0 + i, T) == start + i for i in range(16))   # contiguous
        assert (16 * t) // T == (16 * t + 15) // T                 # one class per chunk
        chunk_sum[t] = cur[start:start + 16].sum()
    incl = np.cumsum(chunk_sum)
    off = incl - chunk_sum
    total = int(incl[-1])
    cbase = np.zeros(17, dtype=np.int64)
    cbase[16] = total
    for t in range(T):
        start = chunk_start(t, T)
        if (16 * t) % T == 0:
            cbase[(16 * t) // T] = off[t]
        run = off[t]
        for i in range(16):
            x = cur[start + i]
            cur[start + i] = run
            run += x
    # scatter
    pos = np.full((T, 16), -1, dtype=np.int64)
    for t in range(T):
        tt = t + 4 * (t // 32)
        for i in range(16):
            q = cls[t, i]
            if q < 0:
                continue
            p = cur[q * Tp + tt]
            cur[q * Tp + tt] = p + 1
            pos[t, i] = p
    got = pos[pos >= 0]
    assert total == len(got) <= STAGE
    assert np.array_equal(np.sort(got), np.arange(total))        # a permutation
    # class order, then thread order, then column order inside a class
    for q in range(16):
        ts, cs = np.nonzero(cls == q)
        order = np.lexsort((cs, ts))
        p_q = pos[ts[order], cs[order]]
        assert np.array_equal(p_q, np.arange(cbase[q], cbase[q] + len(p_q)))
        assert cbase[q + 1] - cbase[q] == len(p_q)
    # bank conflicts: chunk reads (8 lanes per 16-byte phase) and count writes
    rng = np.random.default_rng(T + 1)
    for w in range(nwarps):
        for ph in range(4):
            lanes = [t for t in range(32 * w + 8 * ph, 32 * w + 8 * ph + 8)
                     if (16 * t) // T == (16 * (32 * w + 8 * ph)) // T]     # phases inside one class
            for i in range(4):
                groups = {((chunk_start(t, T) + 4 * i) % 32) // 4 for t in lanes}
                assert len(groups) == len(lanes)
        for _ in range(20):                                         # random class per lane
            qs = rng.integers(0, 16, size=32)
            banks = {cpos(int(qs[l]), 32 * w + l, T) % 32 for l in range(32)}
            assert len(banks) == 32
    return pos, cbase


@pytest.mark.parametrize("T", [640, 672, 800, 896, 1024])
def test_half_tile_random_classes(T):
    rng = np.random.default_rng(T)
    run_half_tile(class_of_columns(rng, T))
    run_half_tile(class_of_columns(rng, T, valid_frac=0.37))


@pytest.mark.parametrize("T", [640, 1024])
def test_half_tile_worst_cases(T):
    # every column in one class; classes by thread; nothing valid; one key
    run_half_tile(np.full((T, 16), 11))
    run_half_tile(np.tile((np.arange(T) % 16)[:, None], (1, 16)))
    run_half_tile(np.full((T, 16), -1))
    one = np.full((T, 16), -1)
    one[T - 1, 15] = 15
    pos, cbase = run_half_tile(one)
    assert pos[T - 1, 15] == 0 and cbase[15] == 0 and cbase[16] == 1
