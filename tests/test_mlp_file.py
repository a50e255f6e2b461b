"""The learned factor's network file (ph_mlp_file_write / ph_mlp_file_read):
the layout documented in include/phpp.h, parsed here independently with
struct, a round trip that keeps every bit, and damaged files refused.  Host
only: no GPU is needed."""
import struct

import numpy as np
import pytest

from paper_1802_09824_gb300 import binding as B


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for c in data:
        h ^= c
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _weights(seed=1):
    return np.random.default_rng(seed).normal(0, 0.5, 321).astype(np.float32)


def test_file_layout_and_round_trip(tmp_path):
    w = _weights()
    w[5] = np.float32(-0.0)
    w[7] = np.float32(1e-40)        # a subnormal keeps its bits too
    path = tmp_path / "g.phmlp"
    B.ph_mlp_file_write(path, w, 0.9765625, 4.39453125, 6.5e-4, 6.8e-9, 400000)
    raw = path.read_bytes()
    assert len(raw) == 1348
    assert raw[:8] == b"PHMLP\x00\x00\x01"
    version, count, rs, rcut, err, loss, steps, res = struct.unpack_from("<IIddffiI", raw, 8)
    assert (version, count, res) == (1, 321, 0)
    assert (rs, rcut, steps) == (0.9765625, 4.39453125, 400000)
    assert err == np.float32(6.5e-4) and loss == np.float32(6.8e-9)
    ws = np.frombuffer(raw, "<f4", 321, 48)
    assert ws.tobytes() == w.tobytes()
    h, res2 = struct.unpack_from("<QQ", raw, 1332)
    assert h == _fnv1a(raw[:1332]) and res2 == 0
    w2, rs2, rcut2, err2, loss2, steps2 = B.ph_mlp_file_read(path)
    assert w2.tobytes() == w.tobytes()
    assert (rs2, rcut2, steps2) == (rs, rcut, steps)
    assert np.float32(err2) == np.float32(6.5e-4) and np.float32(loss2) == np.float32(6.8e-9)


def test_reads_a_file_written_from_the_documented_layout(tmp_path):
    w = _weights(2)
    body = b"PHMLP\x00\x00\x01" + struct.pack("<IIddffiI", 1, 321, 0.5, 2.25, 1e-4, 2e-8, 1234, 0) + w.astype("<f4").tobytes()
    raw = body + struct.pack("<QQ", _fnv1a(body), 0)
    path = tmp_path / "by_hand.phmlp"
    path.write_bytes(raw)
    w2, rs, rcut, err, loss, steps = B.ph_mlp_file_read(path)
    assert w2.tobytes() == w.tobytes() and (rs, rcut, steps) == (0.5, 2.25, 1234)


@pytest.mark.parametrize("damage", ["byte", "truncate", "magic", "version", "count", "longer"])
def test_damaged_files_are_refused(tmp_path, damage):
    path = tmp_path / "g.phmlp"
    B.ph_mlp_file_write(path, _weights(3), 1.0, 4.5, 1e-4, 1e-8, 10)
    raw = bytearray(path.read_bytes())
    if damage == "byte":
        raw[48 + 4 * 100] ^= 0x01            # one weight bit
    elif damage == "truncate":
        raw = raw[:1000]
    elif damage == "magic":
        raw[0] = ord("Q")
    elif damage == "version":
        raw[8] = 2
    elif damage == "count":
        raw[12] = 17
    else:
        raw += b"\x00"
    path.write_bytes(bytes(raw))
    with pytest.raises(B.PhError) as ei:
        B.ph_mlp_file_read(path)
    assert ei.value.code == B.PH_ERR_ARG


def test_missing_file(tmp_path):
    with pytest.raises(B.PhError) as ei:
        B.ph_mlp_file_read(tmp_path / "nothing.phmlp")
    assert ei.value.code == B.PH_ERR_ARG
