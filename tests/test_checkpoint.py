"""Checkpoint file format (host only, no GPU): round trip of the link angles,
trajectory index, parameters and a generator state; refusal of foreign and
truncated files."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1512_03812_gb300 import checkpoint as ck


def _lat():
    L = np.array([8, 4]); T = np.array([6, 4])
    return SimpleNamespace(L=L, T=T, beta=np.array([2.0, 1.5]), m0=np.array([0.1, -0.05]),
                           N=int((L * T).sum()))


def test_round_trip(tmp_path):
    import torch
    lat = _lat()
    rng = np.random.default_rng(5)
    q = rng.uniform(-np.pi, np.pi, (lat.N, 2))
    g = torch.Generator().manual_seed(123)
    torch.randn(7, generator=g)
    path = tmp_path / "a.ckpt"
    ck.save(path, lat, q, 17, rng_state=g.get_state(), params={"scheme": "adapted_nested_fg"})
    c = ck.load(path)
    assert np.array_equal(c["q"], q) and c["q"].dtype == np.float64
    assert c["trajectory"] == 17 and c["params"] == {"scheme": "adapted_nested_fg"}
    assert ck.matches(c, lat)
    g2 = torch.Generator()
    g2.set_state(c["rng_state"])
    assert torch.equal(torch.randn(5, generator=g2), torch.randn(5, generator=g))


def test_refuses_foreign_truncated_and_mismatched(tmp_path):
    lat = _lat()
    q = np.zeros((lat.N, 2))
    path = tmp_path / "b.ckpt"
    ck.save(path, lat, q, 0)
    raw = path.read_bytes()
    (tmp_path / "c.ckpt").write_bytes(b"NOTACKPT" + raw[8:])
    with pytest.raises(ValueError):
        ck.load(tmp_path / "c.ckpt")
    (tmp_path / "d.ckpt").write_bytes(raw[:-8])
    with pytest.raises(ValueError):
        ck.load(tmp_path / "d.ckpt")
    with pytest.raises(ValueError):
        ck.save(tmp_path / "e.ckpt", lat, np.zeros((lat.N, 3)), 0)
    other = _lat()
    other.beta = np.array([2.0, 1.0])
    assert not ck.matches(ck.load(path), other)


def test_failed_save_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    lat = _lat()
    path = tmp_path / "f.ckpt"
    q0 = np.full((lat.N, 2), 0.25)
    ck.save(path, lat, q0, 3)
    before = path.read_bytes()

    def full_disk(fd):
        raise OSError(28, "No space left on device")

    monkeypatch.setattr(ck.os, "fsync", full_disk)
    with pytest.raises(OSError):
        ck.save(path, lat, np.zeros((lat.N, 2)), 4)
    assert path.read_bytes() == before
    assert not (tmp_path / "f.ckpt.tmp").exists()
    assert ck.load(path)["trajectory"] == 3
