"""Host logic of the launch-shape cache (keys, persistence, application to the
options) on the CPU; the GPU name is faked, nothing runs on a device."""
import pytest

from paper_2505_24504_gb300 import autotune, jfnk


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "FAKE GPU")


def _args(nx=20, nz=10, k=2, mu=0.0, prec=32, key=b"mg111111V", periodic=0):
    g = jfnk.Grid(nx, nz, 0.0, 1.0, 0.0, 1.0, periodic)
    ph = jfnk.Physics(1005.0, 717.95, 9.81, 1e5, 300.0, mu, 0, 0.0, 0.0, 0.0)
    o = jfnk.Opts()
    o.precond_prec = prec
    o.mg_key = key
    return g, k, ph, o


def test_keys_separate_every_shape_field(fake_gpu):
    base = autotune.key_of(*_args())
    variants = [_args(nx=40), _args(nz=20), _args(k=3), _args(mu=75.0), _args(prec=64),
                _args(key=b"mg132211V"), _args(periodic=1)]
    keys = {autotune.key_of(*a) for a in variants}
    assert base not in keys and len(keys) == len(variants)
    assert autotune.key_of(*_args()) == base


def test_cache_round_trip_and_apply(tmp_path, fake_gpu):
    path = str(tmp_path / "tune.json")
    assert autotune.load(path) == {}                      # missing file: empty cache
    entry = {"tile_faces": 64, "tile_volume": 1, "tile_fv": 256, "fv_split_cells": 4096}
    autotune.save({autotune.key_of(*_args()): entry}, path)
    got = autotune.load(path)[autotune.key_of(*_args())]
    assert got == entry
    _, _, _, o = _args()
    autotune.apply(o, got)
    assert (o.tile_faces, o.tile_volume, o.tile_fv, o.fv_split_cells) == (64, 1, 256, 4096)
    # entries written before the lane split was tuned leave it at its default
    autotune.apply(o, {"tile_faces": 128, "tile_volume": 2, "tile_fv": 128})
    assert o.fv_split_cells == 0


def test_corrupt_cache_reads_as_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert autotune.load(str(path)) == {}
