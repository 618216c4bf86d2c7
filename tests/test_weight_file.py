"""The learned denoiser's weight file: round trip, flags, and rejection of
damaged files (host logic only)."""
import struct

import numpy as np
import pytest

from paper_1609_04661_gb300 import train_denoiser as td


def test_round_trip_keeps_parameters_and_flag(tmp_path):
    p = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    for scaled in (True, False):
        f = tmp_path / f"w{int(scaled)}.bin"
        td.save_weights(str(f), p, 17, scaled=scaled)
        layers, q, s = td.load_weights(str(f))
        assert layers == 17 and s is scaled
        assert np.array_equal(p, q)


def test_damaged_files_are_rejected(tmp_path):
    p = np.arange(64, dtype=np.float32)
    f = tmp_path / "w.bin"
    td.save_weights(str(f), p, 17, scaled=True)
    raw = bytearray(f.read_bytes())
    bad_magic = tmp_path / "m.bin"
    bad_magic.write_bytes(b"XXXXXXXX" + bytes(raw[8:]))
    flipped = bytearray(raw)
    flipped[40] ^= 1
    bad_crc = tmp_path / "c.bin"
    bad_crc.write_bytes(bytes(flipped))
    short = tmp_path / "s.bin"
    short.write_bytes(bytes(raw[:-4]))
    for g in (bad_magic, bad_crc, short):
        with pytest.raises(ValueError):
            td.load_weights(str(g))


def test_shipped_weights_are_the_full_network():
    layers, params, scaled = td.load_weights()
    c = 64
    expected = 9 * c + c + (layers - 2) * (9 * c * c + c) + 9 * c + 1
    assert layers == 17 and params.size == expected and scaled
    assert np.all(np.isfinite(params))
    assert struct.calcsize("<iiqII") == 24
