"""CPU oracle of the lossless entropy stage — TEST INFRASTRUCTURE ONLY.

Plain Python integers and lists; only the test-suite and the bench's CPU legs may import it.  The
GPU library never does and shares no code with it.

Sec. III-A (its last paragraph) passes the planes and the residual maps that spatial and
temporal coding leave through a lossless coder, Huffman coding being the one it names.

Readings (the paper names the coder and nothing else):
  - The fixed-width frame stream stays the unit of exchange; the entropy stage is a lossless
    transform of it, and its inverse gives back the same bytes.
  - The stream's sections, in order, become: the occupancy bitmap as 8-bit symbols (its bytes);
    the tile codes as 4-bit symbols (one per tile); the run planes and the temporal records
    copied; the fitted bits as 8-bit symbols (its bytes); the residual codes (w_res bits, one per
    fitted pixel) and the raw codes (w_raw bits, one per raw pixel) as symbols of their width.
  - A symbol section of width at most 12 with at least one symbol gets its own Huffman code when
    the coded section (length table, chunk offsets, payload) takes fewer 32-bit words than the
    copy; otherwise it is copied.
  - Code lengths: Huffman's construction over the symbols that occur, sorted by (count, symbol);
    each step joins the two lightest nodes, a leaf before an internal node of equal weight (two
    queues: leaves in sorted order, internal nodes in order of creation).  One symbol alone gets
    length 1.  If a length exceeds 15 every count becomes ceil(count / 2) and the construction
    runs again.
  - Canonical codes: symbols ordered by (length, symbol) take consecutive codes; the first code of
    each length is (first code of the previous length + number of codes of that length) shifted
    left by one, starting from 0 (the canonical rule of DEFLATE).
  - Payload: chunks of 1024 symbols, each starting at a 32-bit word; a code's bits go most
    significant first to increasing bit positions, bit p being bit p % 32 of word p // 32.

Entropy stream layout (little-endian): the fixed-width stream's 64-byte header verbatim; word 16
the magic "LCE1"; word 17 the entropy stream's size in bytes; words 18..45 one descriptor of 4
words per section: (mode | width << 8, count, alphabet, words), mode 0 copy (count = words of the
copy, alphabet 0) or 1 Huffman (count = symbols, alphabet = largest symbol + 1); then the
sections in order.  A Huffman section is its length table (4 bits per symbol of the alphabet,
ceil(alphabet / 8) words), one word per chunk (the chunk's word offset from the payload's start),
then the payload.
"""
from __future__ import annotations

import numpy as np

MAGIC = 0x3145434C        # "LCE1"
FIXED_MAGIC = 0x3143434C  # "LCC1"
CHUNK = 1024
MAX_LEN = 15
MAX_WIDTH = 12
HEADER_WORDS = 16 + 2 + 7 * 4
NAMES = ("bitmap", "tiles", "runs", "temporal", "fitted", "res", "raw")


def _u32(b, off):
    return int.from_bytes(bytes(b[off:off + 4]), "little")


def fixed_layout(fixed: bytes):
    """Per section (name, width or 0 for a copy, symbol count, words) of a fixed-width stream, from
    its header, and the section words."""
    b = bytes(fixed)
    if len(b) < 64 or _u32(b, 0) != FIXED_MAGIC:
        raise ValueError("not a fixed-width stream")
    rows, cols = b[8] | b[9] << 8, b[10] | b[11] << 8
    w_res, w_raw, flags = b[14], b[15], b[7]
    n_tiles, n_runs, n_temp, n_cand, n_fit, n_raw = (_u32(b, o) for o in (24, 32, 36, 40, 44, 48))
    total = _u32(b, 56)

    def words(bits):
        return (bits + 31) // 32

    bw, fw = words(rows * cols), words(n_cand)
    res_w = 0 if flags & 2 else words(n_fit * w_res)
    run_words = (3 if flags & 16 else 4) * n_runs   # three-coefficient planes (flags bit 4): 3 words a run
    secs = [("bitmap", 8, 4 * bw, bw), ("tiles", 4, n_tiles, words(4 * n_tiles)), ("runs", 0, 0, run_words),
            ("temporal", 0, 0, 2 * n_temp), ("fitted", 8, 4 * fw, fw),
            ("res", w_res, 0 if flags & 2 else n_fit, res_w), ("raw", w_raw, n_raw, words(n_raw * w_raw))]
    if 64 + 4 * sum(s[3] for s in secs) != total or total > len(b):
        raise ValueError("inconsistent fixed-width header")
    body = np.frombuffer(b[64:total], "<u4")
    out, o = [], 0
    for name, w, cnt, nw in secs:
        out.append((name, w, cnt, nw, body[o:o + nw].copy()))
        o += nw
    return b[:64], out


def symbols_of(words, width, count):
    """The count fixed-width symbols (LSB-first) held by the words."""
    bits = np.unpackbits(np.asarray(words, "<u4").view(np.uint8), bitorder="little")
    out = []
    for i in range(count):
        v = 0
        for k in range(width):
            v |= int(bits[i * width + k]) << k
        out.append(v)
    return out


def words_of(symbols, width, nwords):
    """Fixed-width symbols (LSB-first) packed into nwords 32-bit words."""
    bits = np.zeros(32 * nwords, np.uint8)
    for i, v in enumerate(symbols):
        for k in range(width):
            bits[i * width + k] = (v >> k) & 1
    return np.packbits(bits, bitorder="little").view("<u4").copy()


def _huffman_depths(used, weight):
    """Leaf depths of Huffman's tree over the used symbols (two queues, a leaf first on ties)."""
    leaves = sorted(used, key=lambda s: (weight[s], s))
    n = len(leaves)
    int_weight, int_parent, leaf_parent = [], [], {}
    li = ii = 0

    def pick():
        nonlocal li, ii
        if li < n and (ii >= len(int_weight) or weight[leaves[li]] <= int_weight[ii]):
            li += 1
            return "leaf", leaves[li - 1], weight[leaves[li - 1]]
        ii += 1
        return "node", ii - 1, int_weight[ii - 1]

    for k in range(n - 1):
        a, b = pick(), pick()
        int_weight.append(a[2] + b[2])
        int_parent.append(None)
        for kind, idx, _ in (a, b):
            if kind == "leaf":
                leaf_parent[idx] = k
            else:
                int_parent[idx] = k
    # the last node made is the root; a node is made after its children, so walk backwards
    depth = [0] * (n - 1)
    for k in range(n - 3, -1, -1):
        depth[k] = depth[int_parent[k]] + 1
    return {s: depth[leaf_parent[s]] + 1 for s in used}


def code_lengths(counts, limit=MAX_LEN):
    """Huffman code length of every symbol (0 where the count is 0), at most limit."""
    counts = [int(c) for c in counts]
    used = [s for s, c in enumerate(counts) if c > 0]
    lengths = [0] * len(counts)
    if not used:
        return lengths
    if len(used) == 1:
        lengths[used[0]] = 1
        return lengths
    weight = {s: counts[s] for s in used}
    while True:
        depth = _huffman_depths(used, weight)
        if max(depth.values()) <= limit:
            break
        weight = {s: (weight[s] + 1) // 2 for s in used}
    for s in used:
        lengths[s] = depth[s]
    return lengths


def first_codes(lengths):
    """First canonical code of every length 1..MAX_LEN (index 0 unused)."""
    per_len = [0] * (MAX_LEN + 1)
    for l in lengths:
        if l:
            per_len[l] += 1
    first, code = [0] * (MAX_LEN + 1), 0
    for l in range(1, MAX_LEN + 1):
        code = (code + per_len[l - 1]) << 1 if l > 1 else 0
        first[l] = code
    return first, per_len


def canonical_codes(lengths):
    first, _ = first_codes(lengths)
    nxt = list(first)
    codes = [0] * len(lengths)
    for s, l in enumerate(lengths):
        if l:
            codes[s] = nxt[l]
            nxt[l] += 1
    return codes


class _BitWriter:
    def __init__(self):
        self.bits = []

    def code(self, c, l):
        for k in range(l - 1, -1, -1):
            self.bits.append((c >> k) & 1)

    def pad(self):
        while len(self.bits) % 32:
            self.bits.append(0)

    def words(self):
        if not self.bits:
            return np.zeros(0, "<u4")
        return np.packbits(np.array(self.bits, np.uint8), bitorder="little").view("<u4").copy()


def _huffman_section(symbols, width):
    """(alphabet, lengths table words, chunk offsets, payload words) of one coded section."""
    alph = max(symbols) + 1
    counts = [0] * alph
    for v in symbols:
        counts[v] += 1
    lengths = code_lengths(counts)
    codes = canonical_codes(lengths)
    table = np.zeros((alph + 7) // 8, "<u4")
    for s, l in enumerate(lengths):
        table[s // 8] |= np.uint32(l << (4 * (s % 8)))
    offsets, payload = [], []
    nwords = 0
    for c0 in range(0, len(symbols), CHUNK):
        w = _BitWriter()
        for v in symbols[c0:c0 + CHUNK]:
            w.code(codes[v], lengths[v])
        w.pad()
        cw = w.words()
        offsets.append(nwords)
        payload.append(cw)
        nwords += len(cw)
    payload = np.concatenate(payload) if payload else np.zeros(0, "<u4")
    return alph, table, np.array(offsets, "<u4"), payload


def encode(fixed: bytes) -> bytes:
    """Entropy stream of a fixed-width frame stream."""
    head, secs = fixed_layout(fixed)
    desc, parts = [], []
    for name, w, cnt, nw, words in secs:
        if w and 0 < cnt and w <= MAX_WIDTH:
            syms = symbols_of(words, w, cnt)
            alph, table, offs, payload = _huffman_section(syms, w)
            hw = len(table) + len(offs) + len(payload)
            if hw < nw:
                desc.append((1 | w << 8, cnt, alph, hw))
                parts.append(np.concatenate([table, offs, payload]))
                continue
        desc.append((0, nw, 0, nw))
        parts.append(words)
    total = 4 * HEADER_WORDS + 4 * sum(d[3] for d in desc)
    hdr = np.frombuffer(head, "<u4").copy()
    ent = np.array([MAGIC, total] + [x for d in desc for x in d], "<u4")
    body = np.concatenate([hdr, ent] + parts).astype("<u4")
    assert 4 * len(body) == total
    return body.tobytes()


def decode(ent: bytes) -> bytes:
    """The fixed-width stream back from its entropy stream; ValueError if it is corrupt."""
    b = bytes(ent)
    if len(b) < 4 * HEADER_WORDS or _u32(b, 64) != MAGIC:
        raise ValueError("bad entropy header")
    total = _u32(b, 68)
    if total > len(b) or total % 4:
        raise ValueError("bad entropy size")
    w32 = np.frombuffer(b[:total], "<u4")
    head = b[:64]
    # expected sections from the fixed header (a zero body of the right size)
    fixed_total = _u32(head, 56)
    if fixed_total < 64 or fixed_total % 4:
        raise ValueError("bad fixed size")
    _, expect = fixed_layout(head + bytes(fixed_total - 64))
    o = HEADER_WORDS
    out = [np.frombuffer(head, "<u4")]
    for s, (name, w, cnt, nw, _) in enumerate(expect):
        mode_w, count, alph, words = (int(x) for x in w32[18 + 4 * s:22 + 4 * s])
        if o + words > len(w32):
            raise ValueError("section overruns the stream")
        sec = w32[o:o + words]
        o += words
        if mode_w == 0:
            if count != nw or words != nw or alph != 0:
                raise ValueError("bad copy descriptor")
            out.append(sec)
            continue
        if mode_w != (1 | w << 8) or not w or w > MAX_WIDTH or count != cnt or alph < 1 or alph > (1 << w):
            raise ValueError("bad Huffman descriptor")
        tw = (alph + 7) // 8
        nch = (count + CHUNK - 1) // CHUNK
        if tw + nch > words:
            raise ValueError("bad Huffman section size")
        lengths = [(int(sec[s_ // 8]) >> (4 * (s_ % 8))) & 15 for s_ in range(alph)]
        kraft = sum(1 << (MAX_LEN - l) for l in lengths if l)
        if kraft > 1 << MAX_LEN or kraft == 0:
            raise ValueError("lengths are not a prefix code")
        first, per_len = first_codes(lengths)
        order = [s_ for l, s_ in sorted((l, s_) for s_, l in enumerate(lengths) if l)]
        index = [0] * (MAX_LEN + 2)
        for l in range(1, MAX_LEN + 1):
            index[l + 1] = index[l] + per_len[l]
        offs = [int(x) for x in sec[tw:tw + nch]]
        pay = sec[tw + nch:]
        bits = np.unpackbits(pay.view(np.uint8), bitorder="little")
        syms = []
        for c in range(nch):
            p = 32 * offs[c]
            end = 32 * (offs[c + 1] if c + 1 < nch else len(pay))
            if p > end or end > len(bits):
                raise ValueError("bad chunk offset")
            for _ in range(min(CHUNK, count - c * CHUNK)):
                code, l = 0, 0
                while True:
                    if p >= end or l >= MAX_LEN:
                        raise ValueError("invalid code")
                    code = code << 1 | int(bits[p])
                    p += 1
                    l += 1
                    if per_len[l] and first[l] <= code < first[l] + per_len[l]:
                        syms.append(order[index[l] + code - first[l]])
                        break
        out.append(words_of(syms, w, nw))
    if o != len(w32):
        raise ValueError("entropy stream size mismatch")
    return np.concatenate(out).astype("<u4").tobytes()
