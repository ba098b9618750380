"""Host model of the Newton-pair schedule (pair variant 3): the index arithmetic of
newton_tile and of the FP64 chunked items, replayed in Python on small ragged
samples.  Every ordered pair (i, j), i != j, of a sample must reach i's sum exactly
once: one-sided inside the block of i's warp, or as a Newton pair (added to one
particle, subtracted, i.e. taken with the opposite sign of d, for the other): between
two warps' blocks of one tile by the cyclic block schedule, or from the tile of the
earlier particle; and the j-side sums must come home to their own lane after the
32-step rotation.  (900, 96, 8) has an odd number of warps, a case no kernel
instantiates, to check the schedule's other branch.
"""
import numpy as np
import pytest


def newton_tile_visits(n, NT, U, base):
    """(i, j, side) visits of the tile starting at `base`, as newton_tile orders them.

    side 'i': pair adds to i one-sided or as the i side of a Newton pair;
    side 'j': the Newton pair's reaction, added to j."""
    W, H = NT // 32, U // 2
    nd = min(n - base, NT * U)                 # the diagonal block
    ngd = -(-nd // 32)

    def i_of(w, h, e, lane):                   # warp w, packed pair h, half e, lane
        return base + w * 32 * U + (2 * h + e) * 32 + lane

    def rotation(G, hs, w, visits):
        # lane l at step k holds j = 32 G + (l + k) % 32 and that j's running sum, which moves
        # to lane l - 1 after the step: follow where each j's sum sits
        holder = {jj: jj for jj in range(32)}
        for k in range(32):
            for lane in range(32):
                jj = (lane + k) % 32
                assert holder[jj] == lane
                j = base + 32 * G + jj
                if j >= n:
                    continue
                for h in hs:
                    for e in range(2):
                        i = i_of(w, h, e, lane)
                        if i < n:
                            visits.append((i, j, "i"))
                            visits.append((j, i, "j"))
            holder = {jj: (hh - 1) % 32 for jj, hh in holder.items()}
        assert all(holder[jj] == jj for jj in range(32))   # home after 32 steps

    visits = []
    # the diagonal block, warp by warp: warp w's i-particles are block B_w (2H groups of 32)
    for w in range(W):
        ival = nd - w * 32 * U
        passes = [(2 * H * w + t, 0) for t in range(2 * H)]                 # own block, one-sided
        for d in range(1, (W - 1) // 2 + 1):                                 # B_{w+d}, Newton pairs
            passes += [(2 * H * ((w + d) % W) + t, "all") for t in range(2 * H)]
        if W % 2 == 0:
            if w < W // 2:       # first H groups of B_{w+W/2}, all packed pairs
                passes += [(2 * H * (w + W // 2) + t, "all") for t in range(H)]
            else:                # every group of B_{w-W/2}, packed pairs h >= H/2
                passes += [(2 * H * (w - W // 2) + t, "upper") for t in range(2 * H)]
        for G, kind in passes:
            if G >= ngd or ival <= (32 * H if kind == "upper" else 0):
                continue
            if kind == 0:
                for lane in range(32):
                    for k in range(32):
                        j = base + 32 * G + k
                        if j - base >= nd:
                            continue
                        for h in range(H):
                            for e in range(2):
                                i = i_of(w, h, e, lane)
                                if i - base < nd and i != j:
                                    visits.append((i, j, "i"))
            else:
                rotation(G, range(H // 2 if kind == "upper" else 0, H), w, visits)
    # the later particles, by j-tiles of NT staged for the whole CTA
    for j0 in range(base + nd, n, NT):
        for w in range(W):
            for g in range(W):
                rotation((j0 - base) // 32 + g, range(H), w, visits)
    return visits


@pytest.mark.parametrize("n,NT,U", [(1500, 64, 8), (2049, 128, 8), (700, 128, 4), (1, 64, 8), (64 * 8, 64, 8),
                                    (1537, 128, 12), (1000, 64, 12), (777, 128, 12), (900, 96, 8)])
def test_every_ordered_pair_once(n, NT, U):
    TI = NT * U
    count = np.zeros((n, n), np.int64)
    for base in range(0, n, TI):
        for a, b, _ in newton_tile_visits(n, NT, U, base):
            count[a, b] += 1
    want = np.ones((n, n), np.int64) - np.eye(n, dtype=np.int64)
    assert np.array_equal(count, want)


def test_sums_match_the_direct_coulomb_sum():
    # the schedule's sums of G(d) = d / max(|d|, dc)^3 weighted by q equal the direct sum (float64)
    rng = np.random.default_rng(0)
    n, NT, U, dc = 777, 64, 8, 0.3
    x = rng.uniform(-5, 5, (n, 3))
    q = rng.uniform(-1, 1, n)

    def G(d):
        r = max(np.linalg.norm(d), dc)
        return d / r ** 3

    acc = np.zeros((n, 3))
    for base in range(0, n, NT * U):
        for a, b, side in newton_tile_visits(n, NT, U, base):
            if side == "i":
                acc[a] += q[b] * G(x[a] - x[b])
            else:       # reaction on the later particle a = j of the pair (b, a): -q_b G(x_b - x_a)
                acc[a] -= q[b] * G(x[b] - x[a])
    ref = np.array([sum(q[j] * G(x[i] - x[j]) for j in range(n) if j != i) for i in range(n)])
    assert np.allclose(acc, ref, rtol=1e-12, atol=1e-12)


def newton_chunks(cap, TI):
    """Chunks per tile of the FP64 Newton-pair items (about 8 tiles of j each, at most 64)."""
    return max(1, min(64, -(-cap // (8 * TI))))


@pytest.mark.parametrize("n,NT", [(6000, 128), (1000, 64), (100000 // 40, 64)])
def test_fp64_chunked_items_cover_each_pair_once(n, NT):
    # item (tile, chunk): j in [max(chunk start, tile start), chunk end); own block one-sided,
    # later particles as Newton pairs; chunks are whole NT-particle j-tiles
    U = 2
    TI = NT * U
    JS = newton_chunks(n, TI)
    ch = -(-(-(-n // JS)) // NT) * NT
    count = np.zeros((n, n), np.int64)
    n_items = 0
    for tile in range(-(-n // TI)):
        base = tile * TI
        dend = min(base + TI, n)
        tile_i = np.arange(base, dend)
        for jc in range(JS):
            cb, ce = jc * ch, min((jc + 1) * ch, n)
            jb = max(cb, base)
            if jb >= ce:
                continue            # the chunk lies before the tile: an empty item
            n_items += 1
            for j0 in range(jb, ce, NT):
                js = np.arange(j0, min(j0 + NT, ce))
                assert (j0 - base) % NT == 0
                if j0 < dend:
                    assert js[-1] < dend or dend == n       # a j-tile never straddles the block's end
                    for i in tile_i:
                        count[i, js[js != i]] += 1
                else:
                    count[np.ix_(tile_i, js)] += 1
                    count[np.ix_(js, tile_i)] += 1
    assert n_items > 0
    want = np.ones((n, n), np.int64) - np.eye(n, dtype=np.int64)
    assert np.array_equal(count, want)
