"""Checkpoint files of the CVAE training state (host side, no GPU): a written state reads back exactly, and a
corrupted, truncated or foreign file is refused rather than resumed from.  Failures are made on the host, by
editing the file's bytes."""
import numpy as np
import pytest

from paper_2011_03082_b300 import checkpoint as ck


def _write(tmp_path, n=1234, **kw):
    rng = np.random.default_rng(3)
    arrs = [rng.standard_normal(n).astype(np.float32) for _ in range(3)]
    path = ck.write(tmp_path / "event.ckpt", name="event", shape=(7, 6, 5, 16), precision=0, step=777, seed=35,
                    lr=1e-3, batch=65536, params=arrs[0], m=arrs[1], v=np.abs(arrs[2]), extra={"log": [[1, 2.5]]},
                    **kw)
    return path, arrs


def test_roundtrip_is_exact(tmp_path):
    path, (p, m, v) = _write(tmp_path)
    st = ck.read(path)
    assert np.array_equal(st["params"], p) and np.array_equal(st["m"], m) and np.array_equal(st["v"], np.abs(v))
    assert (st["name"], st["shape"], st["step"], st["seed"], st["batch"]) == ("event", [7, 6, 5, 16], 777, 35, 65536)
    assert st["lr"] == 1e-3 and st["extra"]["log"] == [[1, 2.5]]
    assert [f.name for f in tmp_path.iterdir()] == ["event.ckpt"]      # no temporary file left behind


@pytest.mark.parametrize("where", ["payload", "header", "crc"])
def test_corruption_is_detected(tmp_path, where):
    path, _ = _write(tmp_path)
    data = bytearray(path.read_bytes())
    off = {"payload": len(data) - 5, "header": ck._FIXED.size + 3, "crc": ck._FIXED.size - 2}[where]
    data[off] ^= 0x10
    path.write_bytes(bytes(data))
    with pytest.raises(ck.CheckpointError, match="CRC|checkpoint"):
        ck.read(path)


def test_truncated_and_foreign_files_are_refused(tmp_path):
    path, _ = _write(tmp_path)
    data = path.read_bytes()
    path.write_bytes(data[:-4])
    with pytest.raises(ck.CheckpointError, match="truncated"):
        ck.read(path)
    path.write_bytes(data[:10])
    with pytest.raises(ck.CheckpointError):
        ck.read(path)
    path.write_bytes(b"NOTACKPT" + data[8:])
    with pytest.raises(ck.CheckpointError, match="not a CVAE checkpoint"):
        ck.read(path)
    bad_version = bytearray(data)
    bad_version[8] = 99
    path.write_bytes(bytes(bad_version))
    with pytest.raises(ck.CheckpointError, match="version"):
        ck.read(path)


def test_mismatched_arrays_are_rejected(tmp_path):
    with pytest.raises(ck.CheckpointError):
        ck.write(tmp_path / "x.ckpt", name="x", shape=(1, 1, 1, 8), precision=0, step=1, seed=1, lr=1e-3, batch=8,
                 params=np.zeros(4, np.float32), m=np.zeros(4, np.float32), v=np.zeros(5, np.float32))
