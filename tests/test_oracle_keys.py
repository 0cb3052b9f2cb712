"""Pins of the oracle's quantisation and sorting keys (CPU only).

Each check ties the oracle to something other than itself: the bit layouts of
Figure 2, closed forms of the quantiser, a textbook 3D Morton code built with a
different algorithm (magic-number bit spreading), and the prefix structure the
paper states for the 20-bit table index (Section 3.1.6).
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure2_layouts.txt")
LO = np.zeros(3, np.float32)
HI = np.ones(3, np.float32)


def figure2_rows():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, *runs = line.split()
            seq = []
            for r in runs:
                seq += [r[0]] * int(r[1:])
            rows[name] = seq
    return rows


def masks_from_row(seq):
    m = {}
    n = len(seq)
    for i, c in enumerate(seq):
        m[c] = m.get(c, 0) | (1 << (n - 1 - i))
    return m


LAYOUTS = {"Aila": oracle.AILA, "Aila_Compact": oracle.AILA_COMPACT, "Two_Point": oracle.TWO_POINT}


def test_golden_rows_have_32_bits():
    rows = figure2_rows()
    assert set(rows) == {"Aila", "Aila_Compact", "Two_Point", "Compact_20", "Origin", "Reis", "Costa",
                         "Octahedron"}
    for name, seq in rows.items():
        assert len(seq) == (20 if name == "Compact_20" else 32), name


@pytest.mark.parametrize("name", ["Aila", "Aila_Compact", "Two_Point", "Compact_20"])
def test_figure2_class_masks(name):
    """All-ones in one component class and zeros elsewhere gives that class's mask."""
    rows = figure2_rows()
    seq = rows[name]
    bits = len(seq)
    layout = oracle.AILA_COMPACT if name == "Compact_20" else LAYOUTS[name]
    masks = masks_from_row(seq)
    ones = 0xFFFFFFFF
    second = "t" if layout == oracle.TWO_POINT else "d"
    # first point (origin) all ones
    k = oracle.interleave(layout, [ones, ones, ones, 0, 0, 0], bits)
    assert k == masks["o"], hex(k)
    # second component all ones: for Aila the components are q(d) >> 3, so the
    # largest possible value is ones >> 3
    comp2 = ones if layout == oracle.TWO_POINT else ones >> 3
    k = oracle.interleave(layout, [0, 0, 0, comp2, comp2, comp2], bits)
    assert k == masks[second], hex(k)
    # the zero slots of the Aila layout stay zero for every input
    if "z" in masks:
        k = oracle.interleave(layout, [ones, ones, ones, ones >> 3, ones >> 3, ones >> 3], bits)
        assert k & masks["z"] == 0
        assert k == masks["o"] | masks["d"]


@pytest.mark.parametrize("name", ["Aila", "Aila_Compact", "Two_Point"])
def test_figure2_single_bit_positions(name):
    """Each single input bit lands where Figure 2 and its x,y,z caption put it.

    Walking the row from the most significant bit, the k-th bit of a class is
    component k mod 3 (x, y, z) of triple k div 3; triples of a class are
    successive levels (bits 31, 30, ... of the quantised coordinate)."""
    seq = figure2_rows()[name]
    layout = LAYOUTS[name]
    count = {}
    for pos, c in enumerate(seq):
        if c == "z":
            continue
        k = count.get(c, 0)
        count[c] = k + 1
        axis = k % 3
        level = k // 3
        if c == "d" and layout in (oracle.AILA, oracle.AILA_COMPACT):
            # direction triples start at level 3 (three leading zero bits)
            level += 3
        comp = [0] * 6
        slot = axis if c == "o" else 3 + axis
        if c == "d":
            comp[slot] = 1 << (31 - level + 3)  # q(d) >> 3 moves bit 34-L to 31-L
            comp[slot] >>= 3
        else:
            comp[slot] = 1 << (31 - level)
        key = oracle.interleave(layout, comp, 32)
        assert key == 1 << (31 - pos), (name, pos, c, hex(key))


def _spread3_10bit(x):
    # textbook 3D Morton bit spreading (magic numbers), 10-bit input
    x &= 0x3FF
    x = (x * 0x00010001) & 0xFF0000FF
    x = (x * 0x00000101) & 0x0F00F00F
    x = (x * 0x00000011) & 0xC30C30C3
    x = (x * 0x00000005) & 0x49249249
    return x


def morton30(x, y, z):
    return (_spread3_10bit(x) << 2) | (_spread3_10bit(y) << 1) | _spread3_10bit(z)


def test_origin_bits_are_textbook_morton():
    """With the second point at zero, the origin bits of the Two Point key are
    the classic 30-bit Morton code of the 10-bit coordinates."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = rng.integers(0, 2**32, size=3, dtype=np.uint64).astype(np.uint32)
        key = oracle.interleave(oracle.TWO_POINT, [q[0], q[1], q[2], 0, 0, 0], 60)
        # gather the origin bits (the first three of every six)
        m = 0
        for L in range(10):
            m = (m << 3) | ((key >> (60 - 6 * L - 3)) & 7)
        assert m == morton30(int(q[0] >> 22), int(q[1] >> 22), int(q[2] >> 22))


def test_longer_keys_extend_shorter_ones():
    """Keys of b bits are prefixes of the 192-bit string: key_b == key_64 >> (64-b)."""
    rng = np.random.default_rng(7)
    for layout in (oracle.AILA, oracle.AILA_COMPACT, oracle.TWO_POINT):
        for _ in range(50):
            comp = rng.integers(0, 2**32, size=6, dtype=np.uint64).astype(np.uint32)
            if layout != oracle.TWO_POINT:
                comp[3:] >>= 3
            k64 = oracle.interleave(layout, comp, 64)
            for b in (1, 16, 20, 31, 32, 33, 48, 63):
                assert oracle.interleave(layout, comp, b) == k64 >> (64 - b)


def test_compact_drops_exactly_the_zero_slots():
    """Aila Compact is the Aila string with its nine always-zero bits removed."""
    rng = np.random.default_rng(9)
    for _ in range(100):
        comp = rng.integers(0, 2**32, size=6, dtype=np.uint64).astype(np.uint32)
        comp[3:] >>= 3
        a = oracle.interleave(oracle.AILA, comp, 64)
        c = oracle.interleave(oracle.AILA_COMPACT, comp, 55)
        # remove bit positions (from MSB, 0-based) 3,4,5, 9,10,11, 15,16,17 of a
        s = format(a, "064b")
        drop = {3, 4, 5, 9, 10, 11, 15, 16, 17}
        kept = "".join(ch for i, ch in enumerate(s) if i not in drop)
        assert int(kept, 2) == c


# ------------------------------------------------------------- quantisation

def test_quantise_closed_forms():
    assert oracle.quantise_unit(0.0) == 0
    assert oracle.quantise_unit(-3.0) == 0
    assert oracle.quantise_unit(float("nan")) == 0
    assert oracle.quantise_unit(1.0) == 0xFFFFFFFF
    assert oracle.quantise_unit(7.0) == 0xFFFFFFFF
    assert oracle.quantise_unit(0.5) == 0x80000000
    assert oracle.quantise_unit(0.25) == 0x40000000
    # the largest float below one maps to 2^32 - 2^8
    assert oracle.quantise_unit(np.nextafter(np.float32(1), np.float32(0))) == 0xFFFFFF00
    lo = np.array([-1, 2, 0], np.float32)
    hi = np.array([1, 6, 8], np.float32)
    assert list(oracle.quantise_point(lo, lo, hi)) == [0, 0, 0]
    assert list(oracle.quantise_point(hi, lo, hi)) == [0xFFFFFFFF] * 3
    assert list(oracle.quantise_point((lo + hi) / 2, lo, hi)) == [0x80000000] * 3
    # outside the box clamps to the faces
    assert list(oracle.quantise_point(hi + 5, lo, hi)) == [0xFFFFFFFF] * 3
    assert list(oracle.quantise_point(lo - 5, lo, hi)) == [0] * 3
    # a degenerate axis quantises to zero
    assert list(oracle.quantise_point([0.3, 0.3, 0.3], [0, 0.3, 0], [1, 0.3, 1]))[1] == 0


def test_quantise_direction_closed_forms():
    assert list(oracle.quantise_direction([1, 0, 0])) == [0xFFFFFFFF, 0x80000000, 0x80000000]
    assert list(oracle.quantise_direction([-1, 0, 0])) == [0, 0x80000000, 0x80000000]
    # normalisation: length does not matter
    assert list(oracle.quantise_direction([0, 0, 5])) == [0x80000000, 0x80000000, 0xFFFFFFFF]
    # zero direction maps to the centre
    assert list(oracle.quantise_direction([0, 0, 0])) == [0x80000000] * 3


def test_largest_extent():
    assert oracle.largest_extent([0, -1, 2], [1, 3, 2.5]) == np.float32(4)


def test_aila_key_of_axis_ray():
    """Origin at the box centre, direction +x: known bits at every level."""
    k = oracle.key(oracle.AILA, 64, [0.5, 0.5, 0.5], [1, 0, 0], 0.0, LO, HI)
    # q(o) = 0x80000000 each; a = (0xFFFFFFFF, 0x80000000, 0x80000000) >> 3
    comp = [0x80000000] * 3 + [0x1FFFFFFF, 0x10000000, 0x10000000]
    assert k == oracle.interleave(oracle.AILA, comp, 64)
    # level 0: o = 111, slots zero; levels 1-2: zero; level 3: bit 28 of every
    # a (the top bit of q(d)); level 4 on: only a_x has ones
    s = format(k, "064b")
    assert s[:36] == "111000" "000000" "000000" "000111" "000100" "000100"


def test_two_point_fixed_equals_given_quarter_extent():
    """Section 3.1.6: the fixed estimate is 0.25 of the largest extent."""
    rng = np.random.default_rng(3)
    lo = np.array([-1, 0, 2], np.float32)
    hi = np.array([3, 1, 4], np.float32)
    E = oracle.largest_extent(lo, hi)
    assert E == np.float32(4)
    o = (lo + rng.random((100, 3)) * (hi - lo)).astype(np.float32)
    d = rng.normal(size=(100, 3)).astype(np.float32)
    ot = np.concatenate([o, np.zeros((100, 1), np.float32)], 1)
    dt = np.concatenate([d, np.full((100, 1), np.inf, np.float32)], 1)
    kf = oracle.compute_keys(oracle.TWO_POINT, 64, ot, dt, lo, hi, tsrc=oracle.T_FIXED, ratio=0.25)
    kg = oracle.compute_keys(oracle.TWO_POINT, 64, ot, dt, lo, hi, tsrc=oracle.T_GIVEN,
                             t_given=np.full(100, 0.25 * 4, np.float32))
    assert np.array_equal(kf, kg)


def test_two_point_termination_point_closed_form():
    """p = o + t*dhat: from the centre along +x by half the width lands on the +x face."""
    lo = np.zeros(3, np.float32)
    hi = np.array([2, 2, 2], np.float32)
    o = np.array([1, 1, 1], np.float32)
    k = oracle.key(oracle.TWO_POINT, 64, o, [3, 0, 0], 1.0, lo, hi)
    comp = [0x80000000] * 3 + [0xFFFFFFFF, 0x80000000, 0x80000000]
    assert k == oracle.interleave(oracle.TWO_POINT, comp, 64)
    # half of that distance: p.x = 1.5 -> 0.75 -> 0xC0000000
    k = oracle.key(oracle.TWO_POINT, 64, o, [3, 0, 0], 0.5, lo, hi)
    comp = [0x80000000] * 3 + [0xC0000000, 0x80000000, 0x80000000]
    assert k == oracle.interleave(oracle.TWO_POINT, comp, 64)
    # a non-finite estimate uses 4*E, which clamps to the face
    k = oracle.key(oracle.TWO_POINT, 64, o, [-1, 0, 0], float("inf"), lo, hi)
    comp = [0x80000000] * 3 + [0, 0x80000000, 0x80000000]
    assert k == oracle.interleave(oracle.TWO_POINT, comp, 64)


def test_table_cell_is_compact_prefix():
    """The 20-bit cell is the 20-bit prefix of the compacted Aila key."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        o = rng.random(3).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        cell = oracle.table_cell(o, d, LO, HI)
        k32 = oracle.key(oracle.AILA_COMPACT, 32, o, d, 0.0, LO, HI)
        assert cell == k32 >> 12
        assert cell < (1 << 20)


# ------------------------------------------------------------- other key families

OD_LAYOUTS = {"Origin": oracle.ORIGIN, "Reis": oracle.REIS, "Costa": oracle.COSTA,
              "Octahedron": oracle.OCTAHEDRON}


def _od_comp(layout, origin, direction):
    """Component vector of or_interleave_od with `origin` / `direction` bits set."""
    if layout == oracle.OCTAHEDRON:
        return [origin] * 3 + [direction >> 4] * 2
    return [origin] * 3 + [direction] * 3


@pytest.mark.parametrize("name", ["Origin", "Reis", "Costa", "Octahedron"])
def test_figure2_class_masks_other_families(name):
    seq = figure2_rows()[name]
    masks = masks_from_row(seq)
    layout = OD_LAYOUTS[name]
    ones = 0xFFFFFFFF
    assert oracle.interleave_od(layout, _od_comp(layout, ones, 0), 32) == masks["o"]
    if "d" in masks:
        assert oracle.interleave_od(layout, _od_comp(layout, 0, ones), 32) == masks["d"]
        assert oracle.interleave_od(layout, _od_comp(layout, ones, ones), 32) == 0xFFFFFFFF


@pytest.mark.parametrize("name", ["Origin", "Reis", "Costa", "Octahedron"])
def test_figure2_single_bit_positions_other_families(name):
    """The k-th o (d) bit of a row is axis k mod 3 (mod 2 for the octahedral
    u, v) at level k div 3 (div 2) of its component; octahedral direction bits
    start at level 4 (four leading zero bits)."""
    seq = figure2_rows()[name]
    layout = OD_LAYOUTS[name]
    count = {}
    for pos, c in enumerate(seq):
        k = count.get(c, 0)
        count[c] = k + 1
        comp = [0] * 6
        if c == "o":
            comp[k % 3] = 1 << (31 - k // 3)
        elif layout == oracle.OCTAHEDRON:
            comp[3 + k % 2] = 1 << (31 - (k // 2 + 4))
        else:
            comp[3 + k % 3] = 1 << (31 - k // 3)
        assert oracle.interleave_od(layout, comp, 32) == 1 << (31 - pos), (name, pos, c)


def test_origin_key_is_textbook_morton():
    rng = np.random.default_rng(21)
    for _ in range(200):
        q = rng.integers(0, 2**32, size=3, dtype=np.uint64).astype(np.uint32)
        k30 = oracle.interleave_od(oracle.ORIGIN, [q[0], q[1], q[2]], 30)
        assert k30 == morton30(int(q[0] >> 22), int(q[1] >> 22), int(q[2] >> 22))


def test_reis_and_costa_split_origin_and_direction():
    """32 bits: Reis = 22 origin + 10 direction bits, Costa = 8 direction + 24 origin."""
    rng = np.random.default_rng(22)
    for _ in range(100):
        c = rng.integers(0, 2**32, size=6, dtype=np.uint64).astype(np.uint32)
        ko22 = oracle.morton3_prefix(c[0], c[1], c[2], 22)
        kd10 = oracle.morton3_prefix(c[3], c[4], c[5], 10)
        assert oracle.interleave_od(oracle.REIS, c, 32) == (ko22 << 10) | kd10
        kd8 = oracle.morton3_prefix(c[3], c[4], c[5], 8)
        ko24 = oracle.morton3_prefix(c[0], c[1], c[2], 24)
        assert oracle.interleave_od(oracle.COSTA, c, 32) == (kd8 << 24) | ko24


def test_octahedral_closed_forms():
    """Poles, equator points and the folded lower hemisphere (Meyer et al. 2010)."""
    cases = {(0, 0, 1): (0.5, 0.5), (0, 0, -1): (1.0, 1.0), (1, 0, 0): (1.0, 0.5), (-1, 0, 0): (0.0, 0.5),
             (0, 1, 0): (0.5, 1.0), (0, -1, 0): (0.5, 0.0), (1, 1, 0): (0.75, 0.75),
             (1, 0, -1): (1.0, 0.75), (-1, 0, -1): (0.0, 0.75), (0, 0, 0): (0.5, 0.5)}
    for d, (u, v) in cases.items():
        uu, vv = oracle.octahedral(np.array(d, np.float32))
        assert (float(uu), float(vv)) == (u, v), d
    # the map is onto the square and scale-free
    rng = np.random.default_rng(23)
    for _ in range(200):
        d = rng.normal(size=3).astype(np.float32)
        u, v = oracle.octahedral(d)
        assert 0.0 <= u <= 1.0 and 0.0 <= v <= 1.0
        u2, v2 = oracle.octahedral(d * np.float32(4.0))
        assert (u, v) == (u2, v2)


def test_other_family_keys_from_rays_use_the_quantisers():
    o = np.array([0.25, 0.5, 0.75], np.float32)
    d = np.array([0, 0, 1], np.float32)
    qo = oracle.quantise_point(o, LO, HI)
    qd = oracle.quantise_direction(d)
    assert oracle.key_od(oracle.ORIGIN, 64, o, d, LO, HI) == oracle.interleave_od(oracle.ORIGIN, qo, 64)
    assert oracle.key_od(oracle.REIS, 48, o, d, LO, HI) == oracle.interleave_od(oracle.REIS, list(qo) + list(qd), 48)
    u, v = oracle.octahedral(d)
    comp = list(qo) + [oracle.quantise_unit(u) >> 4, oracle.quantise_unit(v) >> 4]
    assert oracle.key_od(oracle.OCTAHEDRON, 64, o, d, LO, HI) == oracle.interleave_od(oracle.OCTAHEDRON, comp, 64)
