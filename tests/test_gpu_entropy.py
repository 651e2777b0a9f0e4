"""Entropy stage on the GPU (Sec. III-A, the lossless coder) against its oracle, through the C ABI.

* bit-exact: the entropy stream of an oracle-packed frame stream equals the oracle's, byte for
  byte (lengths, canonical codes, chunk offsets, the copy-or-code choice);
* round trip: the GPU decoder gives back the fixed-width stream, byte for byte, from the GPU's
  and from the oracle's entropy streams; at full size, the sequence the encoder produced decodes
  through the entropy stage to within q/2;
* errors: too small an output latches LCC_ERR_CAPACITY with the needed size; corrupt entropy
  streams latch LCC_ERR_CORRUPT.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import entropy as E
from tests import harness as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06972_gb300 import lcc
    lcc.load()


def _dev(b: bytes, cap=None):
    n = len(b) if cap is None else cap
    t = torch.zeros(max(n, 16), dtype=torch.uint8, device="cuda")
    if b:
        t[:len(b)] = torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()
    return t


def _run(c, fn, streams, caps=None):
    from paper_2008_06972_gb300 import lcc
    n = len(streams)
    caps = caps or [c.max_encoded_bytes + 4096] * n
    d_in = [_dev(s) for s in streams]
    d_out = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for cap in caps]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    fn(d_in, [len(s) for s in streams], d_out, caps, nb)
    st = c.lcc_sync()
    sizes = [int(x) for x in nb.cpu().numpy()]
    outs = [d_out[i][:sizes[i]].cpu().numpy().tobytes() if st == lcc.OK else None for i in range(n)]
    return st, sizes, outs


@pytest.fixture(scope="module")
def oracle_streams(cfg2_seq):
    seq = cfg2_seq
    s, p = O.sensor(seq.sensor), O.params()
    kbits, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
    out = [kbits.tobytes()]
    for f in (0, 3, 9):
        pb, _, _, _ = O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
        out.append(pb.tobytes())
    nd, _, _, _ = O.encode_keyframe(s, O.params(no_delta=1, fit_thr_m=0.02), seq.frames[seq.key_index])
    out.append(nd.tobytes())
    re_, _, _, _ = O.encode_keyframe(s, O.params(raw_exact=1), seq.frames[seq.key_index])
    out.append(re_.tobytes())   # 32-bit raw codes: a copied section
    p3 = O.params(plane3=1)
    k3, kft3, _, _ = O.encode_keyframe(s, p3, seq.frames[seq.key_index])
    out.append(k3.tobytes())    # three-coefficient run records
    pb3, _, _, _ = O.encode_pframe(s, p3, kft3, seq.poses[3], seq.frames[3])
    out.append(pb3.tobytes())
    return out


def test_entropy_streams_match_the_oracle_and_round_trip(cfg2_seq, oracle_streams):
    from paper_2008_06972_gb300 import lcc
    c = H.ctx(cfg2_seq.sensor, max_batch=16)
    st, sizes, ent = _run(c, c.lcc_entropy_encode, oracle_streams)
    assert st == lcc.OK, lcc.status_string(st)
    want = [E.encode(b) for b in oracle_streams]
    for i, (g, w) in enumerate(zip(ent, want)):
        assert sizes[i] == len(w)
        assert g == w, f"stream {i}: entropy stream differs from the oracle's"
        assert len(w) < len(oracle_streams[i])
    st, sizes, back = _run(c, c.lcc_entropy_decode, want)
    assert st == lcc.OK, lcc.status_string(st)
    for i, b in enumerate(back):
        assert b == oracle_streams[i]


@pytest.mark.parametrize("case", ["cfg1_4x4", "cfg1_8x8", "empty", "offgrid_8x16"])
def test_entropy_edge_streams(case):
    from paper_2008_06972_gb300 import lcc
    sensor, pts = synth.frame_cfg1(0)
    s = O.sensor(sensor)
    tile = {"cfg1_4x4": (4, 4), "cfg1_8x8": (8, 8), "empty": (4, 4), "offgrid_8x16": (8, 16)}[case]
    if case == "empty":
        pts = np.zeros((0, 4), np.float32)
    if case == "offgrid_8x16":
        pts = synth.offgrid_points(20000, 5)
    bits, _, _, _ = O.encode_keyframe(s, O.params(*tile), pts)
    fixed = bits.tobytes()
    c = H.ctx(sensor, tile_h=tile[0], tile_w=tile[1])
    st, sizes, ent = _run(c, c.lcc_entropy_encode, [fixed])
    assert st == lcc.OK, lcc.status_string(st)
    assert ent[0] == E.encode(fixed)
    st, _, back = _run(c, c.lcc_entropy_decode, ent)
    assert st == lcc.OK and back[0] == fixed


def test_full_size_sequence_through_the_entropy_stage(cfg2_seq):
    """The GPU-encoded HDL-64E sequence: entropy-encoded and decoded in one call each, the round
    trip is the identity and the frames decode within q/2 of the oracle's range images."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    c = H.ctx(seq.sensor, max_batch=16)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(c)
    c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                          [o.numel() for o in outs], nb, kf)
    assert c.lcc_sync() == lcc.OK
    fixed_sizes = [int(x) for x in nb.cpu().numpy()]
    cap = c.max_encoded_bytes + 4096
    ent = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(n)]
    enb = torch.zeros(n, dtype=torch.int64, device="cuda")
    c.lcc_entropy_encode(outs, [o.numel() for o in outs], ent, [cap] * n, enb)
    assert c.lcc_sync() == lcc.OK
    ent_sizes = [int(x) for x in enb.cpu().numpy()]
    assert sum(ent_sizes) < 0.8 * sum(fixed_sizes)
    back = [torch.zeros(c.max_encoded_bytes, dtype=torch.uint8, device="cuda") for _ in range(n)]
    bnb = torch.zeros(n, dtype=torch.int64, device="cuda")
    c.lcc_entropy_decode(ent, ent_sizes, back, [b.numel() for b in back], bnb)
    assert c.lcc_sync() == lcc.OK
    assert [int(x) for x in bnb.cpu().numpy()] == fixed_sizes
    for f in range(n):
        assert torch.equal(back[f][:fixed_sizes[f]], outs[f][:fixed_sizes[f]])
    # the round-tripped streams decode within q/2 of the input's range image
    s = O.sensor(seq.sensor)
    kfd = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(back[seq.key_index], fixed_sizes[seq.key_index], kfd)
    for f in (seq.key_index, 0, n - 1):
        isk = f == seq.key_index
        rng, _, _ = O.range_image(s, seq.frames[f])
        st, drng, _, _ = H.decode(c, back[f][:fixed_sizes[f]].cpu().numpy(), None if isk else kfd,
                                  None if isk else seq.poses[f])
        assert st == 0
        m = rng > 0
        assert ((drng > 0) == m).all()
        assert np.abs(drng[m] - rng[m]).max() <= 0.01 + 1e-5


def test_capacity_and_corrupt_streams(cfg2_seq, oracle_streams):
    from paper_2008_06972_gb300 import lcc
    c = H.ctx(cfg2_seq.sensor, max_batch=16)
    fixed = oracle_streams[0]
    want = E.encode(fixed)
    st, sizes, _ = _run(c, c.lcc_entropy_encode, [fixed], caps=[len(want) - 16])
    assert st == lcc.ERR_CAPACITY and sizes[0] == len(want)
    st, _, _ = _run(c, c.lcc_entropy_encode, [fixed[:-4]])   # fewer bytes than the header states
    assert st == lcc.ERR_CORRUPT
    bad = bytearray(want)
    bad[64] ^= 1                                             # magic
    st, _, _ = _run(c, c.lcc_entropy_decode, [bytes(bad)])
    assert st == lcc.ERR_CORRUPT
    st, _, _ = _run(c, c.lcc_entropy_decode, [want[:-4]])    # truncated
    assert st == lcc.ERR_CORRUPT
    bad = bytearray(want)
    for i in range(4 * E.HEADER_WORDS, 4 * E.HEADER_WORDS + 8):
        bad[i] = 0x11                                        # lengths that are not a prefix code
    st, _, _ = _run(c, c.lcc_entropy_decode, [bytes(bad)])
    assert st == lcc.ERR_CORRUPT
    bad = bytearray(want)
    hdr = np.frombuffer(want, "<u4")
    o = E.HEADER_WORDS + int(hdr[21])                        # the tile-code section's chunk table
    tw = (int(hdr[24]) + 7) // 8
    assert int(hdr[22]) & 255 == 1
    bad[4 * (o + tw):4 * (o + tw) + 4] = (10 ** 6).to_bytes(4, "little")   # chunk offset past the payload
    st, _, _ = _run(c, c.lcc_entropy_decode, [bytes(bad)])
    assert st == lcc.ERR_CORRUPT
    # the context still works
    st, _, back = _run(c, c.lcc_entropy_decode, [want])
    assert st == lcc.OK and back[0] == fixed
