"""CPU model of the shared-memory exchanges of the register/shared-memory FFT (csrc/fft.cuh).

The 2-D transform of an M x M tile passes data between threads three ways: the line-internal swap
(layout A: line * LDA + k2 * SA + t * ST), the transpose (layout B: x * M + (y ^ hB(x))) and the
twiddle table (t * (E + 1) + k2). The strides are read from the header, so the model follows the
source. For every access the kernels make (virtual thread vt = tid + v * TR, every unrolled loop
index), the model checks:
  * each exchange is a bijection onto slots inside the tile's buffer (nothing overwritten, nothing
    read that was not written, Tile::SMEM slots suffice);
  * a line-internal swap reads only what threads of its own warp wrote (a warp barrier suffices);
  * every half-warp of one 8-byte access touches 16 distinct bank pairs, or shares an address
    (broadcast): no bank conflicts.
Configurations: the fused kernels and the generator (M = 8 ... 64 with one line per thread,
M = 128 with 512 threads x 2 lines) and M = 256 at 512 threads. The staged passes of big.cu
(256- and 512-point lines, 16 threads per line) are modelled the same way: their line swap, twiddle
table and the column passes' staged tile.
"""
import pathlib
import re

import pytest

FFT = pathlib.Path(__file__).resolve().parents[1] / "paper_2406_06640_gb300" / "csrc" / "fft.cuh"


def _ternary(name):
    """Value table of `static constexpr int NAME = M == a ? x : M == b ? y : ... : default;`."""
    src = FFT.read_text()
    m = re.search(r"static constexpr int " + name + r" = (.*?);", src)
    assert m, name
    expr = m.group(1)
    table = {int(a): int(b) for a, b in re.findall(r"M == (\d+) \? (\d+) :", expr)}
    tail = expr.rsplit(":", 1)[1].strip()
    return table, int(tail) if tail.isdigit() else None  # a symbolic default (LDA: E)


SA_T, ST_T, LDA_T = _ternary("SA"), _ternary("ST"), _ternary("LDA")


class Tile:
    def __init__(self, M, sa=None, st=None, lda=None):
        self.M = M
        self.E = min(16, M)
        self.G = M // self.E
        self.T = M * self.G
        self.EG = self.E // self.G
        pick = lambda t: t[0].get(M, t[1])
        self.SA = pick(SA_T) if sa is None else sa
        self.ST = pick(ST_T) if st is None else st
        self.LDA = (LDA_T[0].get(M, self.E)) if lda is None else lda
        self.LDN = M + self.G if self.G > 1 else M + 1
        self.LOG2E = {16: 4, 8: 3}.get(self.E, 0)
        self.S = {16: 4, 8: 3, 4: 2, 2: 1}.get(self.EG, 0)
        self.SMEM = max(M * self.LDA if self.G > 1 else 0, M * M, M * self.LDN)

    def idxA(self, line, t, k2):
        return line * self.LDA + k2 * self.SA + t * self.ST

    def idxB(self, y, x):
        m = (1 << self.S) - 1
        xl = x & (self.E - 1)
        return x * self.M + (y ^ ((xl & ~m) ^ ((xl & m) << (self.LOG2E - self.S))))


def _conflicts(addrs):
    """Bank-conflict count of one 8-byte warp access: per half-warp, lanes at distinct addresses
    must sit in distinct bank pairs (slot mod 16)."""
    n = 0
    for h in range(0, len(addrs), 16):
        half = [a for a in addrs[h:h + 16] if a is not None]
        distinct = set(half)
        n += len(distinct) - len({a % 16 for a in distinct})
    return n


def _accesses(tl, V, TR):
    """Every shared-memory access of fft2_forward / fft2_inverse as (exchange, instruction, tid ->
    slot); an instruction is one unrolled (v, loop indices) combination."""
    E, G, EG = tl.E, tl.G, tl.EG
    out = []

    def per_tid(f):
        return [f(tid) for tid in range(TR)]

    for v in range(V):
        rowmap = lambda tid: divmod(tid + v * TR, G)  # (line, t) or (c, t)
        if G > 1:
            for k2 in range(E):  # swap write (own registers k2)
                out.append(("A-write", (v, k2), per_tid(lambda tid: tl.idxA(*rowmap(tid), k2))))
            for i2 in range(EG):  # swap read (thread tt's register t * EG + i2)
                for tt in range(G):
                    out.append(("A-read", (v, i2, tt), per_tid(
                        lambda tid: tl.idxA(rowmap(tid)[0], tt, rowmap(tid)[1] * EG + i2))))
        for i2 in range(EG):  # transpose, ROW side
            for k1 in range(G):
                out.append(("B-row", (v, i2, k1), per_tid(
                    lambda tid: tl.idxB(rowmap(tid)[0], rowmap(tid)[1] * EG + i2 + E * k1))))
        for j in range(E):  # transpose, COLUMN side: column c, y = t + G j
            out.append(("B-col", (v, j), per_tid(lambda tid: tl.idxB(rowmap(tid)[1] + G * j, rowmap(tid)[0]))))
        if G > 1:
            for k2 in range(1, E):  # twiddle table
                out.append(("W", (v, k2), per_tid(lambda tid: (tid + v * TR) % G * (E + 1) + k2)))
    return out


CONFIGS = [(8, 1), (16, 1), (32, 1), (64, 1), (128, 2), (256, 8)]


@pytest.mark.parametrize("M,V", CONFIGS)
def test_exchanges_are_bijections_inside_the_buffer(M, V):
    tl = Tile(M)
    # layout A over (line, t, k2), layout B over (y, x): injective and inside Tile::SMEM
    if tl.G > 1:
        a = [tl.idxA(l, t, k) for l in range(M) for t in range(tl.G) for k in range(tl.E)]
        assert len(set(a)) == len(a) and min(a) >= 0 and max(a) < tl.SMEM
    b = [tl.idxB(y, x) for y in range(M) for x in range(M)]
    assert len(set(b)) == M * M and min(b) >= 0 and max(b) < tl.SMEM
    # the transpose's two sides visit the same slots
    acc = _accesses(tl, V, tl.T // V)
    row = {s for kind, _, sl in acc if kind == "B-row" for s in sl}
    col = {s for kind, _, sl in acc if kind == "B-col" for s in sl}
    assert row == col == set(b)


@pytest.mark.parametrize("M,V", [c for c in CONFIGS if c[0] >= 32])
def test_line_swaps_stay_inside_a_warp(M, V):
    tl = Tile(M)
    TR = tl.T // V
    writer = {}
    for kind, ins, sl in _accesses(tl, V, TR):
        if kind == "A-write":
            for tid, s in enumerate(sl):
                writer[s] = tid
    for kind, ins, sl in _accesses(tl, V, TR):
        if kind == "A-read":
            for tid, s in enumerate(sl):
                assert writer[s] // 32 == tid // 32, (M, ins, tid, writer[s])


@pytest.mark.parametrize("M,V", CONFIGS)
def test_every_exchange_is_bank_conflict_free(M, V):
    tl = Tile(M)
    TR = tl.T // V
    bad = []
    for kind, ins, sl in _accesses(tl, V, TR):
        for w in range(0, TR, 32):
            c = _conflicts(sl[w:w + 32])
            if c:
                bad.append((kind, ins, w // 32, c))
    assert not bad, bad[:5]


def test_model_sees_a_conflicting_stride():
    """Not vacuous: the M = 128 swap with its row stride one slot longer conflicts."""
    tl = Tile(128, lda=Tile(128).LDA + 1)
    conf = sum(_conflicts(sl[w:w + 32]) for kind, _, sl in _accesses(tl, 2, 512) if kind.startswith("A")
               for w in range(0, 512, 32))
    assert conf > 0


# ---------------------------------------------------------------- staged line transforms (csrc/big_line.cuh)
BIG = FFT.parent / "big_line.cuh"


def _big_shape(BL):
    """LINES and TWS of BigShape<BL>, and the swap row stride BS = BT + 1, read from big_line.cuh."""
    src = BIG.read_text()
    bt = int(re.search(r"constexpr int BT = (\d+);", src).group(1))
    bs = bt + 1
    m = re.search(r"struct BigShape<" + str(BL) + r"> \{\s*static constexpr int (.*?);", src, re.S)
    fields = dict(f.strip().split(" = ") for f in m.group(1).split(","))
    tws = fields["TWS"].strip()
    return int(fields["LINES"]), (bs if tws == "BS" else int(tws)), bt, bs


def _line_freq(BL, t, r):
    return t + 16 * r if BL == 256 else 2 * t + (r >> 4) + 32 * (r & 15)


def _big_accesses(BL):
    """Per 16-thread line (one half-warp): (access, [slot of lane t]) for the swap, the twiddles and the
    column passes' staged tile (natural and frequency order)."""
    LINES, TWS, BT, BS = _big_shape(BL)
    E = 16 if BL == 256 else 32
    TP = LINES + 1
    out = []
    if BL == 256:
        for k2 in range(16):
            out.append(("swap-write", [k2 * BS + t for t in range(BT)]))
        for tt in range(16):
            out.append(("swap-read", [t * BS + tt for t in range(BT)]))
    else:
        for k2 in range(32):
            out.append(("swap-write", [(k2 & 1) * 16 * BS + (k2 >> 1) * BS + t for t in range(BT)]))
        for i2 in range(2):
            for tt in range(16):
                out.append(("swap-read", [i2 * 16 * BS + t * BS + tt for t in range(BT)]))
    for k2 in range(1, E):
        out.append(("twiddle", [t * TWS + k2 for t in range(BT)]))
    for cl in range(LINES):
        for j in range(E):
            out.append(("tile-natural", [(t + 16 * j) * TP + cl for t in range(BT)]))
            out.append(("tile-frequency", [_line_freq(BL, t, j) * TP + cl for t in range(BT)]))
    return out


@pytest.mark.parametrize("BL", [256, 512])
def test_staged_line_swaps_are_bijections(BL):
    LINES, TWS, BT, BS = _big_shape(BL)
    acc = _big_accesses(BL)
    w = [s for kind, sl in acc if kind == "swap-write" for s in sl]
    r = [s for kind, sl in acc if kind == "swap-read" for s in sl]
    assert len(set(w)) == len(w) == BL and set(r) == set(w)
    # the frequencies a line holds after the forward transform are each frequency once
    E = 16 if BL == 256 else 32
    assert sorted(_line_freq(BL, t, q) for t in range(BT) for q in range(E)) == list(range(BL))


@pytest.mark.parametrize("BL", [256, 512])
def test_staged_exchanges_bank_conflicts(BL):
    worst = {}
    for kind, sl in _big_accesses(BL):
        worst[kind] = max(worst.get(kind, 0), _conflicts(sl))
    for kind in ("swap-write", "swap-read", "twiddle", "tile-natural"):
        assert worst[kind] == 0, (BL, kind)
    # frequency order: rows t + 16 r at 256 (conflict-free); rows 2t + i at 512, where lanes t and
    # t + 8 share a bank pair in any [BL][LINES + 1] tile: exactly a 2-way conflict (8 extra per access)
    assert worst["tile-frequency"] == (0 if BL == 256 else 8)
