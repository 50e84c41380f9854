"""The direct-mapped visited cache stores in each slot only the bits of the
hashed id that the slot index does not fix. That is exact only because
id -> (id * odd constant) mod 2^b is a bijection on [0, 2^b): these checks
restate the slot / tag split (as the kernel computes it) on the CPU and
confirm that no two ids below 2^idbits share a (slot, tag) pair, and that the
tag widths the planner picks are the ones the header documents."""
import numpy as np
import pytest

K = 0x9E3779B1


def slot_tag(ids, bits, tag_bits):
    b = bits + tag_bits
    h = (ids.astype(np.uint64) * K) & np.uint64(0xFFFFFFFF)
    if b < 32:
        h &= np.uint64((1 << b) - 1)
    return h >> np.uint64(tag_bits), (h & np.uint64((1 << tag_bits) - 1)) + np.uint64(1)


@pytest.mark.parametrize("idbits,bits", [(10, 8), (15, 8), (15, 12), (17, 8), (17, 10), (20, 14), (20, 12), (12, 14)])
def test_slot_and_tag_name_exactly_one_id(idbits, bits):
    tag_bits = max(0, idbits - bits)
    ids = np.arange(1 << idbits, dtype=np.uint64)
    s, t = slot_tag(ids, bits, tag_bits)
    assert int(s.max()) < (1 << bits)
    assert int(t.min()) >= 1 and int(t.max()) <= (1 << tag_bits)
    pair = s * np.uint64(1 << 16) + t
    assert np.unique(pair).size == ids.size


def test_slots_spread_consecutive_ids():
    # consecutive ids (neighbour lists of a graph are often close in id) land in distinct slots more
    # often than uniformly random slots would (1 - 1/e of 4096 distinct for 4096 random throws)
    s, _ = slot_tag(np.arange(4096, dtype=np.uint64), 12, 8)
    assert np.unique(s).size > 4096 * 0.70
    assert np.unique(s[:1024]).size > 1024 * 0.95


@pytest.mark.parametrize("idbits,bits,width", [(20, 14, 1), (21, 14, 1), (22, 14, 2), (29, 14, 2), (30, 14, 4),
                                               (15, 8, 1), (17, 8, 2)])
def test_slot_width_rule(idbits, bits, width):
    tb = max(0, idbits - bits)
    assert (1 if tb <= 7 else 2 if tb <= 15 else 4) == width
