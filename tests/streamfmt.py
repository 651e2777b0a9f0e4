"""Independent reader of the stream header and fixed-width code sections (test helper).

Layout (little-endian): a 64-byte header, then 32-bit-word sections in this
order: occupancy bitmap (rows*cols bits, raster), tile codes (4 bits per tile),
run planes (4 fp32 words each; with flags bit 4, Eq. 3's three coefficients each, the run start's
tile code 6 + axis naming the dominant axis), temporal records (u32 K-tile index, fp32 c'),
fitted bits (one per candidate pixel), residual codes (w_res bits, k + k_max;
none when flags bit 1, the no-delta mode, is set), raw codes (w_raw bits).  Bits
are LSB-first within words.
"""
import numpy as np

FIELDS = [("magic", 0, "<u4"), ("version", 4, "<u2"), ("kind", 6, "u1"), ("flags", 7, "u1"),
          ("rows", 8, "<u2"), ("cols", 10, "<u2"), ("tile_h", 12, "u1"), ("tile_w", 13, "u1"),
          ("w_res", 14, "u1"), ("w_raw", 15, "u1"), ("thr", 16, "<f4"), ("q", 20, "<f4"),
          ("n_tiles", 24, "<u4"), ("n_valid", 28, "<u4"), ("n_runs", 32, "<u4"),
          ("n_temporal", 36, "<u4"), ("n_cand", 40, "<u4"), ("n_fitted", 44, "<u4"),
          ("n_raw", 48, "<u4"), ("k_max", 52, "<i4"), ("total_bytes", 56, "<u4")]


def header(bits) -> dict:
    b = np.asarray(bits, np.uint8)
    return {name: np.frombuffer(b[off:off + np.dtype(dt).itemsize].tobytes(), dt)[0].item()
            for name, off, dt in FIELDS}


def _words(n_bits):
    return (n_bits + 31) // 32


def sections(bits) -> dict:
    h = header(bits)
    sizes = [("bitmap", _words(h["rows"] * h["cols"])), ("tiles", _words(4 * h["n_tiles"])),
             ("runs", (3 if h["flags"] & 16 else 4) * h["n_runs"]),
             ("temporal", 2 * h["n_temporal"]), ("fitted", _words(h["n_cand"])),
             ("res", 0 if h["flags"] & 2 else _words(h["n_fitted"] * h["w_res"])),
             ("raw", _words(h["n_raw"] * h["w_raw"]))]
    w = np.frombuffer(np.asarray(bits, np.uint8)[64:h["total_bytes"]].tobytes(), "<u4")
    out, o = {}, 0
    for name, n in sizes:
        out[name] = w[o:o + n]
        o += n
    out["header"] = h
    return out


def unpack(words, width, count):
    """Fixed-width LSB-first codes from 32-bit words."""
    bits = np.unpackbits(np.asarray(words, "<u4").view(np.uint8), bitorder="little")
    bits = bits[:width * count].reshape(count, width).astype(np.uint64)
    return (bits << np.arange(width, dtype=np.uint64)).sum(1)


def tile_codes(bits):
    s = sections(bits)
    return unpack(s["tiles"], 4, s["header"]["n_tiles"]).astype(np.uint8)


def residual_codes(bits):
    s = sections(bits)
    h = s["header"]
    return unpack(s["res"], h["w_res"], h["n_fitted"]).astype(np.int64) - h["k_max"]


def raw_codes(bits):
    s = sections(bits)
    h = s["header"]
    return unpack(s["raw"], h["w_raw"], h["n_raw"]).astype(np.int64)
