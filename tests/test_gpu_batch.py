"""Batched ensemble: runs of different shapes, windows, boundary conditions,
viscosities and storage types advanced by one launch per phase evolve bit for
bit as they do alone, for any launch shape; the batch checks its inputs; and a
batched run agrees with the FP64 oracle."""
import numpy as np
import pytest

from paper_2408_15115_gb300 import inputs as I

from cases import TOL_U_F32, gpu_velocity, make_pair, rel_max

pytestmark = pytest.mark.gpu


def _runs():
    """Five runs: closed box (FP32), sliding periodic window with pressure top
    and sponge (FP16), a periodic window as wide as the support box (BF16), a
    mixed-boundary box with the literal rotation update (FP32), and a sliding
    window in BF16 with stochastically rounded stores."""
    from paper_2408_15115_gb300 import turret as T
    out = []
    V, Tr = I.sphere(4, 8.0)
    t = T.Turret(32, 32, 48, 0.05, 2.5, (0, 0, -1e-5), 1, 1, 1, 1)
    t.set_fields(*I.random_state((48, 32, 32), u_amp=0.01, rho_amp=0.001, kmax=3, seed=11))
    t.load_surface(V, Tr, (15.5, 15.7, 30.2))
    out.append(t)
    V, Tr = I.ellipsoid(5, (5.0, 2.5, 2.5))
    V = I.rotate(V, "x", 30.0)
    t = T.Turret(40, 40, 64, 0.03, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=6, slide=1, anchor_frac=0.25,
                 storage="f16")
    t.load_surface(V, Tr, (19.6, 20.3, 16.0), v0=(0, 0, -0.08), w0=(0.001, 0, 0))
    out.append(t)
    V, Tr = I.sphere(4, 9.0)
    t = T.Turret(20, 20, 40, 0.08, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=4, storage="bf16")
    t.load_surface(V, Tr, (9.8, 10.1, 20.5), v0=(0.002, 0, -0.01))
    out.append(t)
    V, Tr = I.ellipsoid(4, (4.0, 3.0, 2.5))
    t = T.Turret(32, 24, 40, 0.04, 3.0, (0, 0, -5e-5), 1, 0, 1, 1, flags={"rot_form": 1})
    t.set_fields(*I.random_state((40, 24, 32), u_amp=0.005, rho_amp=0.0005, kmax=2, seed=12))
    t.load_surface(V, Tr, (15.2, 11.9, 20.0), w0=(0, 0.002, 0.001))
    out.append(t)
    V, Tr = I.sphere(4, 8.0)
    t = T.Turret(24, 24, 48, 0.05, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=4, slide=1, anchor_frac=0.3,
                 storage="bf16", flags={"stochastic_rounding": 1})
    t.load_surface(V, Tr, (11.7, 12.2, 16.0), v0=(0, 0.001, -0.02))
    out.append(t)
    return out


def _snapshot(t):
    s = t.state()
    pops = t.populations().cpu().numpy()
    return s, pops


def _assert_same(a, b):
    sa, pa = a
    sb, pb = b
    for k in ("r", "d", "v", "w", "F", "T", "L", "origin"):
        assert np.array_equal(sa[k], sb[k]), (k, sa[k], sb[k])
    assert sa["step"] == sb["step"]
    assert np.array_equal(pa, pb)


@pytest.fixture(scope="module")
def alone_40():
    runs = _runs()
    for t in runs:
        t.step(40)
    snaps = [_snapshot(t) for t in runs]
    for t in runs:
        t.close()
    return snaps


def test_batched_runs_equal_runs_alone_bitwise(alone_40):
    from paper_2408_15115_gb300 import turret as T
    runs = _runs()
    b = T.Batch(runs)
    b.step(40)
    for t, ref in zip(runs, alone_40):
        _assert_same(_snapshot(t), ref)
    # the sliding run did slide, the narrow window runs without the far/near split
    assert runs[1].state()["origin"][2] <= -1
    b.close()


@pytest.mark.parametrize("threads,minb,tx", [(256, 3, [64, 128, 16, 32, 32]), (64, 2, [32, 64, 16, 64, 16])])
def test_launch_shape_does_not_change_results(alone_40, threads, minb, tx):
    from paper_2408_15115_gb300 import turret as T
    runs = _runs()
    b = T.Batch(runs)
    b.set_tiles(threads, minb, tx)
    b.step(40)
    for t, ref in zip(runs, alone_40):
        _assert_same(_snapshot(t), ref)
    b.close()


def test_batch_and_single_steps_interleave(alone_40):
    from paper_2408_15115_gb300 import turret as T
    runs = _runs()
    b = T.Batch(runs)
    b.step(15)
    for t in runs:
        t.step(10)  # the contexts continue alone from the batched state
    b.step(15)
    for t, ref in zip(runs, alone_40):
        _assert_same(_snapshot(t), ref)
    b.close()


def test_autotune_picks_a_valid_shape_and_caches(tmp_path):
    from paper_2408_15115_gb300 import autotune as AT
    from paper_2408_15115_gb300 import turret as T
    runs = _runs()
    before = [_snapshot(t) for t in runs]
    b = T.Batch(runs)
    cache = str(tmp_path / "tiles.json")
    c1 = b.autotune(cache_path=cache, reps=3)
    assert c1.threads in (128, 256) and c1.minb in (2, 3) and len(c1.tx) == len(runs)
    # timing left every run unchanged
    for t, ref in zip(runs, before):
        _assert_same(_snapshot(t), ref)
    # a second tuning reads the cache and times nothing
    calls = []
    c2 = AT.tune([AT.RunInfo(t.shape[2], t.storage, t.cells, t) for t in runs],
                 timer=lambda *a: calls.append(a) or 1.0, cache_path=cache,
                 device_name=b.torch.cuda.get_device_name(b.device))
    assert calls == [] and (c2.threads, c2.minb, c2.tx) == (c1.threads, c1.minb, c1.tx)
    b.close()


def test_batch_rejects_invalid_run_lists():
    from paper_2408_15115_gb300 import turret as T
    runs = _runs()[:2]
    with pytest.raises(T.TurretError) as e:
        T.Batch([runs[0], runs[0]])
    assert e.value.status == 1
    bare = T.Turret(16, 16, 16, 0.1)
    with pytest.raises(T.TurretError) as e:
        T.Batch([runs[0], bare])
    assert e.value.status == 4
    runs[1].step(1)
    with pytest.raises(T.TurretError) as e:
        T.Batch(runs)
    assert e.value.status == 4
    runs[0].step(1)
    b = T.Batch(runs)
    with pytest.raises(T.TurretError):
        b.set_tiles(128, 2, [48, 32])
    runs[0].step(1)  # one run stepped alone to the other parity: the batch refuses to step
    with pytest.raises(T.TurretError) as e:
        b.step(1)
    assert e.value.status == 4
    b.close()


@pytest.mark.parametrize("force_eval", [0, 1])
def test_batched_run_matches_oracle(force_eval):
    # the closed-box sphere of the FP32 parity suite, advanced inside a batch
    # with a second (FP16) run, against the FP64 oracle after 100 steps; the
    # force on the offset surface (0) or at the markers as printed (1)
    from paper_2408_15115_gb300 import turret as T
    V, Tr = I.sphere(5, 8.0)
    fields = I.random_state((64, 32, 32), u_amp=0.01, rho_amp=0.001, kmax=4, seed=1)
    t, s = make_pair(32, 32, 64, 0.05, (1, 1, 1, 1), kappa=2.5, g=(0, 0, -1e-5), fields=fields,
                     flags={"force_eval": force_eval},
                     particle=(V, Tr, (15.5, 15.5, 44.0), (0, 0, 0), (0, 0, 0)))
    other = _runs()[1]
    b = T.Batch([other, t])
    b.step(100)
    s.step(100)
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < TOL_U_F32
    a, o = t.state(), s.state()
    assert np.abs(a["F"] - o["F"]).max() / np.abs(o["F"]).max() < 1e-4
    assert np.abs(a["v"] - o["v"]).max() / np.abs(o["v"]).max() < 1e-5
    b.close()


def _wide_16bit_runs():
    """16-bit runs whose far cells fill the batched x-pair launch's 64-wide
    tiles: an FP16 sliding window with a sphere and a BF16 one with
    stochastically rounded stores and a tilted ellipsoid (both wide enough for
    the far/near split), and an FP32 run beside them in the other bulk launch."""
    from paper_2408_15115_gb300 import turret as T
    out = []
    V, Tr = I.sphere(4, 8.0)
    t = T.Turret(64, 64, 96, 0.03, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=6, slide=1, anchor_frac=0.3,
                 storage="f16")
    t.load_surface(V, Tr, (31.6, 32.2, 30.4), v0=(0.0, 0.0, -0.05), w0=(0.0, 0.001, 0.0))
    out.append(t)
    V, Tr = I.ellipsoid(5, (5.0, 3.0, 3.0))
    V = I.rotate(V, "x", 25.0)
    t = T.Turret(64, 64, 64, 0.04, 2.0, (0, 0, -1e-4), 0, 0, 1, 2, sponge=4, slide=1, anchor_frac=0.35,
                 storage="bf16", flags={"stochastic_rounding": 1})
    t.load_surface(V, Tr, (32.3, 31.4, 25.0), v0=(0.001, 0.0, -0.04))
    out.append(t)
    V, Tr = I.sphere(4, 8.0)
    t = T.Turret(32, 32, 48, 0.05, 2.5, (0, 0, -1e-5), 1, 1, 1, 1)
    t.load_surface(V, Tr, (15.5, 15.7, 30.2))
    out.append(t)
    return out


def test_batched_16bit_xpair_launch_equals_runs_alone_bitwise():
    # the far cells of the two 16-bit runs go through the batched x-pair
    # launch (64-wide tiles, one-cell code at the boundary planes, the
    # entering plane and the near region); the same runs alone take the
    # single-window x-pair kernel: populations and particle state bit for bit
    from paper_2408_15115_gb300 import turret as T
    alone = _wide_16bit_runs()
    for t in alone:
        t.step(30)
    ref = [_snapshot(t) for t in alone]
    for t in alone:
        t.close()
    runs = _wide_16bit_runs()
    b = T.Batch(runs)
    b.step(30)
    for t, r in zip(runs, ref):
        _assert_same(_snapshot(t), r)
    assert abs(runs[0].state()["origin"][2]) >= 1 and abs(runs[1].state()["origin"][2]) >= 1  # both slid
    b.close()
