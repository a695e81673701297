"""Checkpoint files and step logs (host-side I/O, no GPU): arrays of every
supported type round-trip bit for bit with their meta data, blobs are
16-byte aligned little-endian, and malformed files are rejected."""
import json
import struct

import numpy as np
import pytest

from paper_2106_07687_gb300 import checkpoint as ck


def test_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    arrays = {"state": rng.standard_normal(891 * 3),
              "weights": rng.standard_normal(55954).astype(np.float32),
              "bits": rng.integers(0, 2 ** 16, 77).astype(np.uint16),
              "grid": rng.integers(-5, 5, (3, 4)).astype(np.int32),
              "empty": np.zeros(0)}
    meta = {"config": {"level_solve": 5, "nu": 0.0065}, "t": 1.25}
    p = tmp_path / "a.ck"
    ck.write(p, arrays, meta)
    m, back = ck.read(p)
    assert m == meta
    assert set(back) == set(arrays)
    for k, a in arrays.items():
        assert back[k].dtype == a.dtype and back[k].shape == a.shape
        assert back[k].tobytes() == a.tobytes()


def test_layout_is_little_endian_and_aligned(tmp_path):
    p = tmp_path / "b.ck"
    ck.write(p, {"x": np.array([1.0, -2.0]), "y": np.array([3], dtype=np.int32),
                 "z": np.array([0.5], dtype=np.float32)})
    data = p.read_bytes()
    assert data[:8] == b"DNNMGCK1"
    (hlen,) = struct.unpack("<I", data[8:12])
    head = json.loads(data[12:12 + hlen])
    base = 12 + hlen
    for e in head["arrays"]:
        assert e["offset"] % 16 == 0 and e["dtype"].startswith("<")
    x = head["arrays"][0]
    assert struct.unpack("<2d", data[base + x["offset"]:base + x["offset"] + 16]) == (1.0, -2.0)


def test_malformed_files_are_rejected(tmp_path):
    p = tmp_path / "c.ck"
    p.write_bytes(b"NOTACKPT" + b"\0" * 8)
    with pytest.raises(ValueError):
        ck.read(p)
    ck.write(p, {"x": np.arange(10.0)})
    data = p.read_bytes()
    p.write_bytes(data[:-24])                       # truncated blob
    with pytest.raises(ValueError):
        ck.read(p)
    with pytest.raises(ValueError):
        ck.write(tmp_path / "d.ck", {"c": np.zeros(2, dtype=np.complex128)})


def test_step_log(tmp_path):
    p = tmp_path / "steps.jsonl"
    with ck.StepLog(p) as log:
        for n in range(3):
            log.write(n, {"newton_its": 3, "gmres_its": 10 + n, "fallback": 0}, t=0.005 * (n + 1))
    rows = ck.read_log(p)
    assert [r["step"] for r in rows] == [0, 1, 2]
    assert rows[2]["gmres_its"] == 12 and rows[1]["t"] == pytest.approx(0.01)
