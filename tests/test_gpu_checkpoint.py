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


def test_tampered_sizes_and_flags_are_refused(tmp_path):
    # a checkpoint whose part sizes do not match the context, or whose
    # rigid-body flags differ, is refused before anything is copied into the
    # workspace; the context stays usable
    import ctypes as C

    from paper_2408_15115_gb300 import turret as T

    class Header(C.Structure):
        _fields_ = [("magic", C.c_char * 8), ("version", C.c_int32), ("storage", C.c_int32),
                    ("has_particle", C.c_int32), ("nm", C.c_int32), ("win", T.Window), ("flags", T.Flags),
                    ("nu", C.c_double), ("kappa", C.c_double), ("g", C.c_double * 3), ("step", C.c_int64),
                    ("nbox", C.c_int64), ("bytes_pop", C.c_int64), ("bytes_utop", C.c_int64),
                    ("bytes_state", C.c_int64), ("bytes_h", C.c_int64), ("bytes_hl", C.c_int64)]

    path = tmp_path / "ck.bin"
    a = _make("f32")
    a.step(3)
    a.save(str(path))
    raw = path.read_bytes()
    h0 = Header.from_buffer_copy(raw[:C.sizeof(Header)])
    assert h0.magic == b"TURRETCK" and h0.nm == a.state()["n_markers"]
    for field in ("bytes_utop", "bytes_h", "bytes_hl"):
        h = Header.from_buffer_copy(raw[:C.sizeof(Header)])
        setattr(h, field, getattr(h, field) + 4096)
        bad = tmp_path / ("bad_%s.bin" % field)
        bad.write_bytes(bytes(h) + raw[C.sizeof(Header):] + b"\0" * 4096)
        with pytest.raises(T.TurretError) as e:
            a.load(str(bad))
        assert e.value.status == 4, field
    c = configs.ensemble_member("prolate", 10.0, 30.0, (64, 64, 64), "f32", seed=3)
    for flag in ("renorm_orientation", "fixed_position"):
        b = configs.make_turret(c, flags={flag: 1})
        b.load_surface(c["verts"], c["tris"], c["r0"], v0=(0, 0, -0.05))
        with pytest.raises(T.TurretError) as e:
            b.load(str(path))
        assert e.value.status == 4, flag
        b.close()
    # the refused loads left the context as it was
    before = a.state()
    a.step(2)
    assert a.state()["step"] == before["step"] + 2
