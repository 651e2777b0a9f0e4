"""The entropy-stage oracle (Sec. III-A, the lossless coder after spatial and temporal coding)
pinned to textbook values, brute force, the Kraft and entropy bounds, and round trips of real
frame streams.  No GPU needed."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle import entropy as E


def _cost(counts, lengths):
    return sum(c * l for c, l in zip(counts, lengths))


def test_textbook_six_letter_example():
    """The classic six-letter frequency table (45, 13, 12, 16, 9, 5): lengths 1, 3, 3, 3, 4, 4 and
    224 bits in all."""
    counts = [45, 13, 12, 16, 9, 5]
    lengths = E.code_lengths(counts)
    assert lengths == [1, 3, 3, 3, 4, 4]
    assert _cost(counts, lengths) == 224


@pytest.mark.parametrize("seed", range(12))
def test_lengths_are_optimal_by_brute_force(seed):
    """No prefix code (Kraft sum <= 1) over up to 6 symbols has a smaller total length."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 7))
    counts = [int(x) for x in rng.integers(1, 60, n)]
    best = min(_cost(counts, ls) for ls in itertools.product(range(1, n), repeat=n)
               if sum(2.0 ** -l for l in ls) <= 1.0)
    assert _cost(counts, E.code_lengths(counts)) == best


@pytest.mark.parametrize("seed", range(8))
def test_codes_are_complete_prefix_free_and_canonical(seed):
    rng = np.random.default_rng(100 + seed)
    alph = int(rng.integers(2, 300))
    counts = [int(x) if rng.random() < 0.7 else 0 for x in rng.geometric(0.05, alph)]
    if sum(1 for c in counts if c) < 2:
        counts[0], counts[1] = 3, 5
    lengths = E.code_lengths(counts)
    codes = E.canonical_codes(lengths)
    used = [s for s, c in enumerate(counts) if c]
    assert all(lengths[s] > 0 for s in used) and all(lengths[s] == 0 for s in range(alph) if not counts[s])
    # Kraft equality: the tree is full
    assert sum(2 ** (E.MAX_LEN - lengths[s]) for s in used) == 2 ** E.MAX_LEN
    # prefix-free
    words = [format(codes[s], f"0{lengths[s]}b") for s in used]
    for a, b in itertools.combinations(words, 2):
        assert not a.startswith(b) and not b.startswith(a)
    # canonical: in (length, symbol) order the codes count up, shifting left when the length grows
    order = sorted(used, key=lambda s: (lengths[s], s))
    assert codes[order[0]] == 0
    for a, b in zip(order, order[1:]):
        assert codes[b] == (codes[a] + 1) << (lengths[b] - lengths[a])
    assert codes[order[-1]] == 2 ** lengths[order[-1]] - 1
    # entropy bound of an unlimited Huffman code
    tot = sum(counts)
    H = -sum(c / tot * math.log2(c / tot) for c in counts if c)
    L = _cost(counts, lengths) / tot
    if max(lengths) < E.MAX_LEN:
        assert H - 1e-12 <= L < H + 1


def test_length_limit_halves_the_counts():
    """Fibonacci counts give a 25-deep tree; the limit halves the counts (rounding up) until the
    depth is at most 15, and the code stays complete."""
    fib = [1, 1]
    while len(fib) < 26:
        fib.append(fib[-1] + fib[-2])
    assert max(E.code_lengths(fib, limit=64)) == 25
    lengths = E.code_lengths(fib)
    assert max(lengths) <= E.MAX_LEN
    assert sum(2 ** (E.MAX_LEN - l) for l in lengths) == 2 ** E.MAX_LEN
    w = list(fib)
    while max(E.code_lengths(w, limit=64)) > E.MAX_LEN:
        w = [(c + 1) // 2 for c in w]
    assert lengths == E.code_lengths(w, limit=64)


def test_single_symbol_gets_one_bit():
    assert E.code_lengths([0, 0, 7, 0]) == [0, 0, 1, 0]
    assert E.canonical_codes([0, 0, 1, 0]) == [0, 0, 0, 0]


def test_ties_take_the_leaf_first():
    """Four equal counts: leaves are joined pairwise first (all lengths 2), not chained."""
    assert E.code_lengths([5, 5, 5, 5]) == [2, 2, 2, 2]
    # counts 1, 1, 2, 2: after the first join the node of weight 2 ties with both leaves of
    # weight 2; taking the leaves first joins them together (all lengths 2), taking the node first
    # would give 3, 3, 2, 1 (the same 12 bits: ties change the lengths, not the cost)
    assert E.code_lengths([1, 1, 2, 2]) == [2, 2, 2, 2]
    # equal counts queue in symbol order: symbols 0 and 1 join first, so symbol 2 gets the 1-bit code
    assert E.code_lengths([1, 1, 1]) == [2, 2, 1]
    assert E.code_lengths([3, 0, 3, 3, 0]) == [2, 0, 2, 1, 0]


@pytest.fixture(scope="module")
def streams():
    seq = synth.sequence_cfg2(0, 3)
    s, p = O.sensor(seq.sensor), O.params()
    kbits, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
    pbits, _, _, _ = O.encode_pframe(s, p, kft, seq.poses[0], seq.frames[0])
    nd = O.params(no_delta=1, fit_thr_m=0.02)
    nbits, _, _, _ = O.encode_keyframe(s, nd, seq.frames[seq.key_index])
    c1, pts1 = synth.frame_cfg1(0)
    s1 = O.sensor(c1)
    b8, _, _, _ = O.encode_keyframe(s1, O.params(8, 8), pts1)
    empty, _, _, _ = O.encode_keyframe(s1, O.params(), np.zeros((0, 4), np.float32))
    return {"key": kbits, "p": pbits, "no_delta": nbits, "cfg1_8x8": b8, "empty": empty}


@pytest.mark.parametrize("name", ["key", "p", "no_delta", "cfg1_8x8", "empty"])
def test_round_trip_of_frame_streams(streams, name):
    fixed = streams[name].tobytes()
    ent = E.encode(fixed)
    assert E.decode(ent) == fixed
    hdr = np.frombuffer(ent, "<u4")
    assert hdr[16] == E.MAGIC and hdr[17] == len(ent)
    if name != "empty":
        assert len(ent) < len(fixed)
    # a copied section is its fixed words; a coded one holds the lengths of its symbols' histogram
    # and one word-padded chunk of codes per 1024 symbols
    _, secs = E.fixed_layout(fixed)
    o = E.HEADER_WORDS
    for k, (nm, w, cnt, nw, words) in enumerate(secs):
        mode, count, alph, size = (int(x) for x in hdr[18 + 4 * k:22 + 4 * k])
        sec = hdr[o:o + size]
        o += size
        if mode & 255 == 0:
            assert count == nw and size == nw and np.array_equal(sec, words)
            continue
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:w * cnt].reshape(cnt, w)
        syms = (bits.astype(np.int64) << np.arange(w)).sum(1)
        hist = np.bincount(syms)
        assert alph == len(hist)
        lengths = np.array([(int(sec[i // 8]) >> (4 * (i % 8))) & 15 for i in range(alph)])
        assert np.array_equal(lengths > 0, hist > 0)
        assert lengths.tolist() == E.code_lengths(hist.tolist())
        nch = (cnt + E.CHUNK - 1) // E.CHUNK
        per_chunk = [int(lengths[syms[c:c + E.CHUNK]].sum()) for c in range(0, cnt, E.CHUNK)]
        assert size == (alph + 7) // 8 + nch + sum((b + 31) // 32 for b in per_chunk)
    assert o == len(hdr)


def test_sections_take_the_smaller_form(streams):
    """A coded section is smaller than its copy; the copy is kept otherwise (the empty frame)."""
    for name in ("key", "empty"):
        fixed = streams[name].tobytes()
        hdr = np.frombuffer(E.encode(fixed), "<u4")
        _, secs = E.fixed_layout(fixed)
        for k, (nm, w, cnt, nw, _) in enumerate(secs):
            mode, words = int(hdr[18 + 4 * k]) & 255, int(hdr[21 + 4 * k])
            assert words <= nw
            if mode == 1:
                assert words < nw


def test_corrupt_entropy_streams_are_rejected(streams):
    ent = bytearray(E.encode(streams["key"].tobytes()))
    with pytest.raises(ValueError):
        E.decode(bytes(ent[:-4]))
    bad = bytearray(ent)
    bad[64] ^= 1
    with pytest.raises(ValueError):
        E.decode(bytes(bad))
    # a length table that is not a prefix code (every symbol of the bitmap's alphabet at length 1)
    hdr = np.frombuffer(bytes(ent), "<u4")
    assert int(hdr[18]) & 255 == 1
    bad = bytearray(ent)
    for i in range(E.HEADER_WORDS * 4, E.HEADER_WORDS * 4 + 8):
        bad[i] = 0x11
    with pytest.raises(ValueError):
        E.decode(bytes(bad))


def _batched_depths(used, weight):
    """Leaf depths of Huffman's two-queue construction taken a batch of joins at a time (the GPU
    builder's schedule, restated here to check that it is exact): with m the weight of the next
    node to be made, every remaining node made so far and every remaining leaf of weight <= m
    is picked before any node made later, so those items, in pick order, pair up at once; an odd
    last item stays at the front of its queue."""
    import bisect
    leaves = sorted(used, key=lambda s: (weight[s], s))
    n = len(leaves)
    lw = [weight[s] for s in leaves]
    nw = [0] * (n - 1)
    leaf_parent, node_parent = [None] * n, [None] * (n - 1)
    li = ni = nk = 0
    big = 1 << 62
    while nk + 1 < n:
        l0 = lw[li] if li < n else big
        l1 = lw[li + 1] if li + 1 < n else big
        n0 = nw[ni] if ni < nk else big
        n1 = nw[ni + 1] if ni + 1 < nk else big
        m = l0 + (l1 if l1 <= n0 else n0) if l0 <= n0 else n0 + (l0 if l0 <= n1 else n1)
        a = bisect.bisect_right(lw, m, li, n) - li
        b = nk - ni
        T, P = a + b, (a + b) // 2
        picked = [None] * T
        for e in range(T):
            if e < a:   # a leaf goes after the nodes strictly lighter than it
                r = e + bisect.bisect_left(nw, lw[li + e], ni, nk) - ni
            else:       # a node goes after the leaves no heavier than it
                r = (e - a) + bisect.bisect_right(lw, nw[ni + e - a], li, li + a) - li
            picked[r] = e
        for r in range(2 * P):
            e = picked[r]
            if e < a:
                leaf_parent[li + e] = nk + r // 2
            else:
                node_parent[ni + e - a] = nk + r // 2
        for q in range(P):
            w = [lw[li + picked[2 * q + k]] if picked[2 * q + k] < a else nw[ni + picked[2 * q + k] - a] for k in (0, 1)]
            nw[nk + q] = w[0] + w[1]
        if T % 2 and picked[T - 1] < a:
            li, ni = li + a - 1, ni + b
        elif T % 2:
            li, ni = li + a, ni + b - 1
        else:
            li, ni = li + a, ni + b
        nk += P
    depth = [0] * (n - 1)
    for k in range(n - 3, -1, -1):
        depth[k] = depth[node_parent[k]] + 1
    return {s: depth[leaf_parent[i]] + 1 for i, s in enumerate(leaves)}


def test_batched_construction_is_the_two_queue_construction():
    """Taking the joins a batch at a time gives every leaf the depth of the one-at-a-time
    two-queue construction (ties included): uniform, geometric, Fibonacci and random count
    tables up to 4096 symbols."""
    rng = np.random.default_rng(11)
    tables = [[1] * 100, [2 ** k for k in range(20)], [1, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144]]
    for _ in range(300):
        n = int(rng.choice([2, 3, 5, 17, 300, 4096]))
        kind = rng.integers(4)
        if kind == 0:
            c = rng.integers(1, 10, n)
        elif kind == 1:
            c = rng.exponential(100.0, n).astype(int) + 1
        elif kind == 2:
            c = (1000 * 2.0 ** -np.abs(rng.normal(0, 3, n))).astype(int) + 1
        else:
            c = rng.choice([1, 2, 3, 5, 8], n)
        tables.append([int(x) for x in c])
    for c in tables:
        used = list(range(len(c)))
        weight = {s: c[s] for s in used}
        assert _batched_depths(used, weight) == E._huffman_depths(used, weight)
