"""Host-side pins of the SSOR block kernel's schedule (qcd_sap_plan_tables; no GPU needed).

The schedule is checked against facts derived here, independently of the planner: the ll
order from the oracle (Sec. 3), the block's nearest-neighbour relation from coordinates, and
the data each site update reads (its in-block neighbours) and writes (itself).

* levels: every in-block neighbour that comes earlier in the ll order sits on a lower level
  and every later one on a higher level (so a level-by-level sweep reads what the sequential
  sweep reads), and levels are as low as that allows (longest-chain levels);
* chunks: each chunk holds one level, chunks follow the level order, no CTA has more than
  nslot sites in a chunk;
* ownership: every site has one owner and one slab offset, offsets are unique per CTA and
  below the slab size, and (warp form) every level is dealt evenly over the CTAs;
* barriers: over three consecutive sweeps of the timeline (forward chunk c at step c,
  backward at 2 nchunks - 1 - c, periodic flags, the set-up barrier before step 0), every
  read of a neighbour's value is separated from the neighbour's previous and next write by
  a barrier: a cluster barrier (2) when the two sites have different owners, at least a CTA
  barrier (1) otherwise.
"""
import numpy as np
import pytest

import oracle
import paper_1210_7398_gb300 as q

GEOMS = [
    ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6)),   # the 12^3 x 24 configuration
    ((12, 12, 12, 24), (6, 6, 6, 6), (3, 3, 3, 3)),    # the paper's 6^4 / 3^4 split
    ((12, 12, 12, 24), (3, 3, 3, 6), (1, 1, 1, 2)),
    ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2)),
    ((24, 24, 24, 48), (4, 4, 4, 4), (2, 2, 2, 2)),
    ((4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 1, 1)),
    ((12, 12, 12, 24), (6, 6, 6, 12), (6, 6, 6, 12)),  # natural order
]


def neighbour_pairs(b):
    """Unordered in-block nearest-neighbour pairs (i, j), block-local lexicographic indices."""
    vol = int(np.prod(b))
    y = np.array(np.unravel_index(np.arange(vol), b, order="F")).T
    out = []
    stride = 1
    for m in range(4):
        i = np.nonzero(y[:, m] + 1 < b[m])[0]
        out.append(np.stack([i, i + stride], axis=1))
        stride *= b[m]
    return np.concatenate(out)


def ll_key(b, s):
    order = oracle.ll_order(b, s)
    key = np.empty(len(order), dtype=np.int64)
    key[order] = np.arange(len(order))
    return key


def check_schedule(b, s, t):
    vol, C, nch, nslot = t["vol"], t["ctas"], t["chunks"], t["nslot"]
    lev, own, slot, ch, fl = t["level"], t["owner"], t["slot"], t["chunk"], t["flags"].astype(np.int64)
    assert vol == int(np.prod(b))
    pairs = neighbour_pairs(b)
    key = ll_key(b, s)
    # levels: ordered like the ll keys along every neighbour pair, and longest-chain minimal
    i, j = pairs[:, 0], pairs[:, 1]
    first = np.where(key[i] < key[j], i, j)
    second = np.where(key[i] < key[j], j, i)
    assert np.all(lev[first] < lev[second])
    need = np.zeros(vol, dtype=np.int64)
    np.maximum.at(need, second, lev[first] + 1)
    assert np.array_equal(lev, need)
    assert lev.max() + 1 == t["levels"]
    # chunks: one level each, in level order, all levels covered; per CTA at most nslot sites
    assert ch.min() == 0 and ch.max() == nch - 1
    chunk_level = np.full(nch, -1)
    for c in range(nch):
        lv = np.unique(lev[ch == c])
        assert len(lv) == 1
        chunk_level[c] = lv[0]
    assert np.all(np.diff(chunk_level) >= 0)
    assert set(chunk_level) == set(range(t["levels"]))
    counts = np.zeros((nch, C), dtype=np.int64)
    np.add.at(counts, (ch, own), 1)
    assert counts.max() == nslot
    # ownership: owners in range, unique slab offsets per CTA, levels dealt evenly
    assert own.min() >= 0 and own.max() < C
    assert slot.min() >= 0 and slot.max() < t["slab_vol"]
    assert len(set(zip(own.tolist(), slot.tolist()))) == vol
    if not t["thread"] and C > 1:
        per = np.zeros((t["levels"], C), dtype=np.int64)
        np.add.at(per, (lev, own), 1)
        assert np.all(per.max(axis=1) - per.min(axis=1) <= 1)
    # barriers: positions 0 .. 3P - 1 over three sweeps; the set-up barrier before position 0
    P = 2 * nch
    pos = np.arange(3 * P)
    strength = fl[pos % P].copy()
    strength[0] = 2
    cum = [np.concatenate([[0], np.cumsum(strength >= k)]) for k in (1, 2)]  # cum[k-1][p + 1]: barriers <= p

    def has_barrier(lo, hi, k):
        # a barrier of strength >= k at some position p with lo < p <= hi (lo = -1: none before)
        c = cum[k - 1]
        return c[hi + 1] - c[lo + 1] > 0

    def writes(site):
        sw = np.arange(3)[None, :] * P
        return np.sort(np.concatenate([sw + ch[site][:, None], sw + P - 1 - ch[site][:, None]], axis=1), axis=1)

    for reader, src in ((i, j), (j, i)):
        k = np.where(own[reader] != own[src], 2, 1)
        wr, ws = writes(reader), writes(src)  # (npairs, 6)
        for col in range(6):
            tt = wr[:, col:col + 1]
            prev = np.where(ws < tt, ws, -1).max(axis=1)
            nxt = np.where(ws > tt, ws, np.iinfo(np.int64).max).min(axis=1)
            t0 = tt[:, 0]
            for kk in (1, 2):
                sel = k == kk
                assert np.all(has_barrier(prev[sel], t0[sel], kk)), "read after write without a barrier"
                has_next = sel & (nxt < np.iinfo(np.int64).max)
                assert np.all(has_barrier(t0[has_next], nxt[has_next], kk)), "write after read without a barrier"


@pytest.mark.parametrize("half", [False, True], ids=["f32", "f16"])
@pytest.mark.parametrize("ctas", [0, 1, 2, 3, 8, 16, -1, -2])
@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: "x".join(map(str, g[1])) + "/" + "x".join(map(str, g[2])))
def test_ssor_schedule_is_consistent(geom, ctas, half):
    dims, b, s = geom
    try:
        t = q.qcd_sap_plan_tables(dims, b, s, sap_ctas=ctas, half=half, sms=152)
    except q.QcdError:
        # a fixed width whose shared memory does not fit is rejected; the automatic one never is
        assert ctas not in (0, -1, -2)
        return
    if ctas >= 1:
        assert t["ctas"] >= ctas
    if ctas == -1:
        assert t["thread"] == (0 if half else t["thread"])
    if ctas == -2:
        # the tile form holds one right-hand side's block spinor (plus 4 zero slots, 2 with FP32
        # storage) in one CTA, with FP16 storage its source as well (12 words per site each, 24
        # for an FP32 spinor), else the automatic cluster form stands in
        vol = int(np.prod(b))
        size = (2 * vol + 4) * 48 if half else (vol + 2) * 96
        fits = size <= 200 * 1024
        assert t["thread"] == (2 if fits else 0)
        if fits:
            assert t["ctas"] == 1 and t["chunks"] == t["levels"]
            assert t["smem_bytes"] == size
    check_schedule(b, s, t)


def test_automatic_width_on_gb300():
    """The widths the kernels run with on 152 SMs: 8 CTAs per 6^3 x 12 block on 12^3 x 24 (8
    blocks per colour), one per block where the blocks of one colour fill the GPU."""
    t = q.qcd_sap_plan_tables((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), sms=152)
    assert (t["ctas"], t["levels"], t["nslot"]) == (8, 12, 26)
    t = q.qcd_sap_plan_tables((24, 24, 24, 48), (4, 4, 4, 4), (2, 2, 2, 2), sms=152)
    assert t["ctas"] == 1
    t = q.qcd_sap_plan_tables((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), sap_ctas=-1, sms=152)
    assert t["ctas"] >= 1  # the thread form does not fit a 2592-site block: the warp form stands in


def test_rejected_geometry():
    with pytest.raises(q.QcdError):
        q.qcd_sap_plan_tables((12, 12, 12, 24), (4, 4, 4, 4), (2, 2, 2, 2))  # 3 blocks along x
    with pytest.raises(q.QcdError):
        q.qcd_sap_plan_tables((12, 12, 12, 24), (6, 6, 6, 12), (4, 3, 3, 6))  # sub-block does not divide


def random_geometries(n, seed=7):
    """Seeded sample of block / sub-block shapes (extents 1..6, sub-blocks dividing them) on
    lattices of two blocks per direction."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        b = [int(rng.integers(1, 7)) for _ in range(4)]
        if np.prod(b) < 2 or np.prod(b) > 1296:
            continue
        s = [int(rng.choice([d for d in range(1, bm + 1) if bm % d == 0])) for bm in b]
        out.append((tuple(2 * bm for bm in b), tuple(b), tuple(s)))
    return out


@pytest.mark.parametrize("geom", random_geometries(24), ids=lambda g: "x".join(map(str, g[1])) + "/" + "x".join(map(str, g[2])))
@pytest.mark.parametrize("ctas,half", [(0, False), (3, False), (0, True), (-1, False), (-2, True)])
def test_ssor_schedule_random_shapes(geom, ctas, half):
    dims, b, s = geom
    try:
        t = q.qcd_sap_plan_tables(dims, b, s, sap_ctas=ctas, half=half, sms=152)
    except q.QcdError:
        assert ctas not in (0, -1, -2)
        return
    check_schedule(b, s, t)


@pytest.mark.parametrize("C", [2, 4, 8, 16])
def test_dealing_keeps_sub_blocks_on_one_cta(C):
    """The sites of a level come in ll order (local position, then sub-block), so dealing them
    round-robin over C CTAs, C dividing the sub-block count, gives sub-block sigma to CTA
    sigma mod C: most neighbour reads stay in the CTA's own shared memory."""
    b, s = (6, 6, 6, 12), (3, 3, 3, 6)
    t = q.qcd_sap_plan_tables((12, 12, 12, 24), b, s, sap_ctas=C, sms=152)
    assert t["ctas"] == C
    vol = int(np.prod(b))
    y = np.array(np.unravel_index(np.arange(vol), b, order="F")).T
    nq = [b[m] // s[m] for m in range(4)]
    sigma = np.ravel_multi_index(tuple((y // np.array(s)).T), nq, order="F")
    assert np.array_equal(t["owner"], sigma % C)
    pairs = neighbour_pairs(b)
    remote = np.mean(t["owner"][pairs[:, 0]] != t["owner"][pairs[:, 1]])
    assert remote < 0.2
