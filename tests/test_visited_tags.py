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


# ----------------------------------------------------- set-associative cache
# visited_mode 4: 2^bits sets of one 32-bit word holding W fields of
# tag_bits + 1 bits, newest lowest; an insert that misses shifts the word up
# one field and puts the tag in the lowest. Restated here as the kernel
# computes it, and checked against a plain model (a list per set, first in
# first out) on random insert sequences.

def ways_for(idbits, bits):
    fw = max(0, idbits - bits) + 1
    return 3 if fw <= 10 else (2 if fw <= 16 else 0)


def assoc_insert(words, bits, tag_bits, W, uid):
    s, t = (int(v[0]) for v in slot_tag(np.array([uid], np.uint64), bits, tag_bits))
    fw = tag_bits + 1
    fmask = (1 << fw) - 1
    wmask = 0xFFFFFFFF if W * fw >= 32 else (1 << (W * fw)) - 1
    old = words[s]
    if any(((old >> (w * fw)) & fmask) == t for w in range(W)):
        return 0
    words[s] = ((old << fw) | t) & wmask
    return 3 if (old >> ((W - 1) * fw)) & fmask else 1


@pytest.mark.parametrize("idbits,bits", [(20, 12), (21, 12), (15, 8), (17, 10), (22, 12), (27, 12)])
def test_assoc_cache_equals_a_fifo_model(idbits, bits):
    W = ways_for(idbits, bits)
    assert W in (2, 3)
    tag_bits = max(0, idbits - bits)
    assert W * (tag_bits + 1) <= 32
    r = np.random.default_rng(idbits * 100 + bits)
    pool = r.integers(0, 1 << idbits, size=(1 << bits) // 2 * 3)  # revisits make hits
    seq = r.choice(pool, size=8 * (1 << bits))
    words = [0] * (1 << bits)
    model = {}
    for u in seq.tolist():
        s = int(slot_tag(np.array([u], np.uint64), bits, tag_bits)[0][0])
        lst = model.setdefault(s, [])
        if u in lst:
            want = 0
        else:
            want = 3 if len(lst) == W else 1
            lst.insert(0, u)
            del lst[W:]
        assert assoc_insert(words, bits, tag_bits, W, u) == want
    # the words decode to exactly the model's ids (no field ever names an id that was not inserted)
    for s, lst in model.items():
        fw = tag_bits + 1
        fields = [(words[s] >> (w * fw)) & ((1 << fw) - 1) for w in range(W)]
        tags = [int(slot_tag(np.array([u], np.uint64), bits, tag_bits)[1][0]) for u in lst]
        assert fields[:len(tags)] == tags and all(f == 0 for f in fields[len(tags):])


@pytest.mark.parametrize("idbits,bits,ways", [(20, 12, 3), (21, 12, 3), (22, 12, 2), (27, 12, 2), (28, 12, 0),
                                              (24, 12, 2), (15, 8, 3)])
def test_assoc_ways_rule(idbits, bits, ways):
    assert ways_for(idbits, bits) == ways
