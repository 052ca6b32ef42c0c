"""The re-rank's two summation schedules give the same bits (CPU emulation).

The exact re-rank sums a Dot2 (compensated) dot product per lane over the
positions t = lane, lane + 32, ... in increasing order, then merges the 32
lane partials by a fixed xor butterfly.  For a sparse row it steps only over
the positions where x_i is nonzero, and it reduces four candidates at once by
a butterfly whose first two levels each keep half of them.  Both rest on two
facts of IEEE single precision, emulated here operation by operation:
a Dot2 step with a zero product leaves (s, c) unchanged, and the
reduce-scatter applies the same merges to the same operands.  TwoProd's FMA
is exact in double: a product of two floats has at most 48 significant bits,
and its rounding error is a float.
"""
import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    z = f32(s - a)
    e = f32(f32(a - f32(s - z)) + f32(b - z))
    return s, e


def dot2_step(s, c, x, y):
    p = f32(x * y)
    ep = f32(np.float64(x) * np.float64(y) - np.float64(p))  # fmaf(x, y, -p)
    t, es = two_sum(s, p)
    return t, f32(c + f32(es + ep))


def dot2_merge(s, c, s2, c2):
    t, e = two_sum(s, s2)
    return t, f32(f32(c + c2) + e)


def butterfly(parts):
    """dot2_warp_reduce: every lane ends with the same (s, c)."""
    parts = list(parts)
    for off in (16, 8, 4, 2, 1):
        nxt = []
        for lane in range(32):
            lo, hi = (lane, lane ^ off) if not lane & off else (lane ^ off, lane)
            nxt.append(dot2_merge(*parts[lo], *parts[hi]))
        parts = nxt
    return parts[0]


def reduce_scatter4(parts4):
    """dot2_reduce4: parts4[u][lane]; lane L ends with candidate 2*bit4 + bit3."""
    def merge_ordered(mine, other, upper):
        return dot2_merge(*other, *mine) if upper else dot2_merge(*mine, *other)

    kept = []
    for lane in range(32):  # level 16: keep {0,1} or {2,3}
        h16 = bool(lane & 16)
        pair = (2, 3) if h16 else (0, 1)
        kept.append([merge_ordered(parts4[u][lane], parts4[u][lane ^ 16], h16) for u in pair])
    cur = []
    for lane in range(32):  # level 8: keep one of the pair
        h8 = bool(lane & 8)
        q = 1 if h8 else 0
        cur.append(merge_ordered(kept[lane][q], kept[lane ^ 8][q], h8))
    for off in (4, 2, 1):
        cur = [merge_ordered(cur[lane], cur[lane ^ off], bool(lane & off)) for lane in range(32)]
    return cur


def lane_partials_dense(a, b):
    out = []
    for lane in range(32):
        s = c = f32(0)
        for t in range(lane, a.size, 32):
            s, c = dot2_step(s, c, a[t], b[t])
        out.append((s, c))
    return out


def lane_partials_sparse(a, b):
    out = []
    for lane in range(32):
        s = c = f32(0)
        for t in range(lane, a.size, 32):
            if a[t] != 0:
                s, c = dot2_step(s, c, a[t], b[t])
        out.append((s, c))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_sparse_steps_and_reduce_scatter_match_dense_butterfly(seed):
    rng = np.random.default_rng(seed)
    d = 300 + 37 * seed
    a = np.zeros(d, np.float32)
    nz = rng.choice(d, int(rng.integers(1, 40)), replace=False)
    a[nz] = rng.standard_normal(nz.size).astype(np.float32) * np.float32(10.0) ** rng.integers(-3, 3, nz.size)
    bs = []
    for u in range(4):
        b = rng.standard_normal(d).astype(np.float32)
        b[rng.random(d) < 0.5] = 0.0      # sparse candidates too
        if u == 3:
            b[nz[: nz.size // 2]] = -a[nz[: nz.size // 2]]   # cancellation
        bs.append(b)
    dense = [butterfly(lane_partials_dense(a, b)) for b in bs]
    sparse_parts = [lane_partials_sparse(a, b) for b in bs]
    for u in range(4):
        assert lane_partials_sparse(a, bs[u]) == lane_partials_dense(a, bs[u])
    rs = reduce_scatter4(sparse_parts)
    for lane in range(32):
        u = 2 * ((lane >> 4) & 1) + ((lane >> 3) & 1)
        assert rs[lane] == dense[u], (lane, u)
