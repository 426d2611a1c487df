"""The checkpoint file format (host only): round trips with and without L-bar,
and every malformed file is refused with CheckpointError."""
import numpy as np
import pytest

from paper_2512_05749_gb300 import checkpoint as ck


def state(M=300, r=16, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((M, r)).astype(np.float32), np.sort(rng.random(r))[::-1], rng.standard_normal(r)


@pytest.mark.parametrize("with_lbar", [False, True])
def test_round_trip_is_exact(tmp_path, with_lbar):
    V, s, L = state()
    p = str(tmp_path / "c.bin")
    ck.save(p, 41, V, s, L if with_lbar else None, rng_counter=2 ** 40 + 3)
    d = ck.load(p)
    assert d["step"] == 41 and d["rng_counter"] == 2 ** 40 + 3
    assert d["V"].dtype == np.float32 and np.array_equal(d["V"], V)
    assert np.array_equal(d["sigma"], s)
    assert (d["Lbar"] is None) == (not with_lbar)
    if with_lbar:
        assert np.array_equal(d["Lbar"], L)


def test_layout_is_the_documented_one(tmp_path):
    V, s, _ = state(M=3, r=2)
    p = str(tmp_path / "c.bin")
    ck.save(p, 7, V, s)
    raw = open(p, "rb").read()
    assert raw[:8] == b"WSSRCKPT"
    assert len(raw) == 8 + 4 + 4 + 8 * 4 + 4 * 6 + 8 * 2 + 8
    assert np.array_equal(np.frombuffer(raw, "<f4", 6, 48).reshape(3, 2), V)


def test_damaged_files_are_refused(tmp_path):
    V, s, L = state()
    p = str(tmp_path / "c.bin")
    ck.save(p, 1, V, s, L)
    raw = bytearray(open(p, "rb").read())
    cases = {"flip": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:], "truncated": raw[:-9],
             "magic": b"XSSRCKPT" + raw[8:], "short": raw[:20]}
    for name, data in cases.items():
        q = str(tmp_path / f"{name}.bin")
        open(q, "wb").write(bytes(data))
        with pytest.raises(ck.CheckpointError):
            ck.load(q)


def test_bad_shapes_are_refused(tmp_path):
    V, s, L = state()
    with pytest.raises(ck.CheckpointError):
        ck.save(str(tmp_path / "a.bin"), 0, V, s[:-1])
    with pytest.raises(ck.CheckpointError):
        ck.save(str(tmp_path / "b.bin"), 0, V, s, L[:3])
    with pytest.raises(ck.CheckpointError):
        ck.save(str(tmp_path / "c.bin"), 0, V[:, 0], s)
