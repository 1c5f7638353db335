"""Checkpoint files (host side of the library, no GPU): round trip, the
CRC-32 of the links against zlib's, and rejection of damaged files."""
import struct
import zlib

import numpy as np
import pytest

from paper_1805_03560_gb300 import hmc


def _field(L, seed=1):
    rng = np.random.default_rng(seed)
    V = int(np.prod(L))
    return rng.normal(size=(V, 4, 3, 3)) + 1j * rng.normal(size=(V, 4, 3, 3))


INFO = dict(L=[4, 2, 2, 6], beta=5.6, kappa=0.1575, seed=2**63 + 5, trajectory=17,
            rng_counter=18, plaquette=0.5712345678901234)


def test_round_trip(tmp_path):
    U = _field(INFO["L"])
    p = str(tmp_path / "a.ckpt")
    hmc.write_checkpoint(p, INFO, U)
    info, U2 = hmc.read_checkpoint(p)
    assert info == INFO
    assert U2.tobytes() == U.tobytes()
    info_only, none = hmc.read_checkpoint(p, links=False)
    assert none is None and info_only == INFO


def test_layout_and_crc(tmp_path):
    U = _field(INFO["L"], 2)
    p = tmp_path / "b.ckpt"
    hmc.write_checkpoint(str(p), INFO, U)
    raw = p.read_bytes()
    assert raw[:8] == b"HMCCKPT1"
    assert list(struct.unpack_from("<4i", raw, 8)) == INFO["L"]
    beta, kappa, seed, traj, ctr, plaq = struct.unpack_from("<2d3Qd", raw, 24)
    assert (beta, kappa, seed, traj, ctr, plaq) == (INFO["beta"], INFO["kappa"], INFO["seed"],
                                                    INFO["trajectory"], INFO["rng_counter"],
                                                    INFO["plaquette"])
    (crc,) = struct.unpack_from("<I", raw, 72)
    assert crc == zlib.crc32(raw[80:]) == zlib.crc32(U.tobytes())
    assert len(raw) == 80 + U.nbytes


def test_damaged_files_rejected(tmp_path):
    U = _field(INFO["L"], 3)
    p = tmp_path / "c.ckpt"
    hmc.write_checkpoint(str(p), INFO, U)
    raw = bytearray(p.read_bytes())
    bad = tmp_path / "flip.ckpt"
    raw[80 + 1000] ^= 0x10
    bad.write_bytes(bytes(raw))
    for links in (True, False):
        with pytest.raises(hmc.HmcError):
            hmc.read_checkpoint(str(bad), links=links)
    short = tmp_path / "short.ckpt"
    short.write_bytes(p.read_bytes()[:-8])
    with pytest.raises(hmc.HmcError):
        hmc.read_checkpoint(str(short))
    magic = tmp_path / "magic.ckpt"
    magic.write_bytes(b"NOTACKPT" + p.read_bytes()[8:])
    with pytest.raises(hmc.HmcError):
        hmc.read_checkpoint(str(magic))
    with pytest.raises(hmc.HmcError):
        hmc.read_checkpoint(str(tmp_path / "missing.ckpt"))


def test_buffer_size_checked(tmp_path):
    U = _field(INFO["L"], 4)
    p = str(tmp_path / "d.ckpt")
    hmc.write_checkpoint(p, INFO, U)
    import ctypes
    ci = hmc.CheckpointInfo()
    buf = np.empty(10, np.float64)
    st = hmc.lib().hmc_checkpoint_read(None, p.encode(), ctypes.byref(ci), buf.ctypes.data, 10)
    assert st == hmc.EINVAL
