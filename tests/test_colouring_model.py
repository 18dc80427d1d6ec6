"""An executable model of the device's colouring scheme, checked against the
oracle's sequential greedy colouring (CPU only).

Every row is a clique of the column-intersection graph, so in the greedy
order the units of a row are coloured one after the other.  The device's
data-flow rounds therefore let a unit wait only for its predecessor in each
of its rows, keep per row a 128-bit mask of the colours its coloured prefix
holds (the last bit standing for "a colour >= 127", which sends the unit to a
slow path that reads the prefix itself), and let the second unit of a
two-unit row read the first one's colour directly.  This model runs those
rounds serially and must give exactly the oracle's colouring -- on random
LPs with dense rows (well past 127 colours), simplex blocks with two columns
in one row, two-unit rows, and on the VC / IS / MC standard forms."""
import numpy as np
import pytest

from paper_1311_2661_gb300 import synth

OVF = 127  # mask bit: a colour >= 127 in the prefix


def _mask_bits(c):
    c = int(c)  # Python integers: the mask is 128 bits wide
    return 1 << (c if c < OVF else OVF)


def _pick(mask):
    if mask >> OVF & 1:
        return -1
    free = ~mask & ((1 << OVF) - 1)
    return (free & -free).bit_length() - 1 if free else -1


def row_chain_colouring(lp, seed):
    """(colour per unit, number of rounds, largest frontier)."""
    e = lp.export()
    us, ul, _ = lp.units()
    U = lp.U
    rank = np.empty(U, np.int64)
    rank[lp.priority_order(seed)] = np.arange(U)
    uoc = np.full(lp.N, -1, np.int64)
    for u in range(U):
        uoc[us[u]:us[u] + ul[u]] = u
    members = [[] for _ in range(lp.M)]
    for j in range(lp.N):
        if uoc[j] >= 0:
            for q in range(e["colptr"][j], e["colptr"][j + 1]):
                members[e["rowidx"][q]].append(int(uoc[j]))
    # a unit repeated in a row (two columns of one block) counts once
    chains = [sorted(set(m), key=lambda u: rank[u]) for m in members]
    links = [[] for _ in range(U)]
    for i, ch in enumerate(chains):
        for pos, u in enumerate(ch):
            links[u].append((i, pos))
    cnt = [sum(pos > 0 for _, pos in links[u]) for u in range(U)]
    mask = [0] * lp.M
    colour = np.full(U, -1, np.int64)
    frontier = [u for u in range(U) if cnt[u] == 0]
    rounds, widest = 0, 0
    while frontier:
        rows_busy = set()
        for u in frontier:  # units of one frontier share no row
            for i, _ in links[u]:
                assert i not in rows_busy
                rows_busy.add(i)
        nxt = []
        for u in frontier:
            m = 0
            for i, pos in links[u]:
                if pos == 0:
                    continue
                m |= _mask_bits(colour[chains[i][0]]) if len(chains[i]) == 2 else mask[i]
            c = _pick(m)
            if c < 0:  # slow path: the colours of the row prefixes themselves
                held = {int(colour[w]) for i, pos in links[u] for w in chains[i][:pos]}
                c = 0
                while c in held:
                    c += 1
            colour[u] = c
            for i, pos in links[u]:
                if pos + 1 < len(chains[i]):
                    if len(chains[i]) != 2:
                        mask[i] |= _mask_bits(c)
                    w = chains[i][pos + 1]
                    cnt[w] -= 1
                    if cnt[w] == 0:
                        nxt.append(w)
        widest = max(widest, len(frontier))
        frontier = nxt
        rounds += 1
    assert np.all(colour >= 0)
    return colour, rounds, widest


def _random_lp(oracle_mod, seed, dense=2, dense_len=180):
    rng = np.random.default_rng(seed)
    n, k = 260, 3
    bf = np.array([10, 100, 200], np.int64)
    rows = [rng.choice(n, dense_len, replace=False) for _ in range(dense)]
    rows += [rng.choice(n, 2, replace=False) for _ in range(60)]
    rows += [np.array([10, 11, 100, 101]), np.array([200, 202, 7]), np.array([12, 10, 150])]
    while len(rows) < 200:
        rows.append(rng.choice(n, int(rng.integers(3, 7)), replace=False))
    M = len(rows)
    entries = sorted((int(j), i) for i, r in enumerate(rows) for j in r)
    colptr = np.zeros(n + 1, np.int64)
    for j, _ in entries:
        colptr[j + 1] += 1
    colptr = np.cumsum(colptr)
    rowidx = np.array([i for _, i in entries], np.int32)
    val = rng.choice([-1.0, 1.0, 2.0], size=len(entries))
    lo = np.zeros(n)
    hi = np.ones(n)
    hi[5] = 0.0  # a fixed column
    rk = rng.integers(0, 3, M).astype(np.uint8)
    return oracle_mod.OracleLP.general(M, colptr, rowidx, val, rng.normal(size=M), rng.normal(size=n), lo, hi, rk,
                                       k, bf)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_model_equals_greedy_past_the_masks(oracle_mod, seed):
    lp = _random_lp(oracle_mod, seed)
    col_o, nc = lp.color(seed)
    assert nc > 150  # dense rows: colours far past the 127 a mask holds
    col_m, rounds, _ = row_chain_colouring(lp, seed)
    assert np.array_equal(col_m, col_o)
    assert rounds > 150  # a chain along each dense row


@pytest.mark.parametrize("kind,mk", [
    ("vc", lambda: synth.er_graph(400, 1600, 1)),
    ("is", lambda: synth.chung_lu(600, 3000, 2.1, 2)),
    ("mc", lambda: synth.grid_graph(12, 9, 3, 3)),
])
def test_model_equals_greedy_on_the_workload_forms(oracle_mod, kind, mk):
    g = mk()
    if kind != "mc":
        g.w = np.ones(g.n, np.float32)
    lp = oracle_mod.build_problem(kind, g)
    col_o, _ = lp.color(5)
    col_m, rounds, widest = row_chain_colouring(lp, 5)
    assert np.array_equal(col_m, col_o)
    assert widest > 1 and rounds < lp.U  # rounds run many units in parallel
