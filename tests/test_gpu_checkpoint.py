"""Checkpoint and resume: a context saved at a time level and restored into
a fresh, identically configured context continues bit for bit; mismatched
configurations and foreign files are refused."""
import numpy as np
import pytest

from paper_2408_15115_gb300 import configs

pytestmark = pytest.mark.gpu


def _make(storage="f32", predictor=None):
    c = configs.ensemble_member("prolate", 10.0, 30.0, (64, 64, 64), storage, seed=3)
    t = configs.make_turret(c)
    if predictor:
        t.set_predictor(predictor, warm=True)
    t.load_surface(c["verts"], c["tris"], c["r0"], v0=(0, 0, -0.05))
    return t


@pytest.mark.parametrize("storage,predictor", [("f32", None), ("f16", "linear")])
def test_resume_is_bitwise(tmp_path, storage, predictor):
    path = str(tmp_path / "ck.bin")
    a = _make(storage, predictor)
    a.step(37)  # odd time level, the window has slid
    a.save(path)
    a.step(25)
    b = _make(storage, predictor)
    b.load(path)
    assert b.state()["step"] == 37
    b.step(25)
    sa, sb = a.state(), b.state()
    for k in ("r", "d", "v", "w", "F", "T", "L", "origin"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["origin"][2] <= -1
    assert np.array_equal(a.populations().cpu().numpy(), b.populations().cpu().numpy())


def test_mismatched_checkpoints_are_refused(tmp_path):
    from paper_2408_15115_gb300 import turret as T
    path = str(tmp_path / "ck.bin")
    a = _make("f32")
    a.step(3)
    a.save(path)
    other = _make("f16")
    with pytest.raises(T.TurretError) as e:
        other.load(path)
    assert e.value.status == 4
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a checkpoint" * 20)
    with pytest.raises(T.TurretError) as e:
        a.load(str(junk))
    assert e.value.status == 1
