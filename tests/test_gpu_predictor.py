"""The force/torque predictor (surrogate modes): the device trajectory log
and the training pairs built from it against the oracle's features, linear
extrapolation and the network's in-step prediction against their
definitions, the fallback rule, drag and settling against the paper's step,
the batched form, and the gain of the trained network over linear
extrapolation on held-out runs."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2408_15115_gb300 import configs
from paper_2408_15115_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _turret(kind="prolate", seed=1, d=12.0, re=20.0, storage="f32"):
    c = configs.ensemble_member(kind, d, re, (64, 64, 64), storage, seed=seed)
    return configs.make_turret(c), c


def _load(t, c):
    t.load_surface(c["verts"], c["tris"], c["r0"])


def test_log_and_training_pairs_vs_oracle():
    from paper_2408_15115_gb300 import turret as T
    t, c = _turret()
    t.set_log(64)
    _load(t, c)
    t.step(40)
    rec = t.log_records()
    assert rec.shape == (41, M.LOG_REC)
    r = rec.cpu().numpy()
    assert np.array_equal(r[:, 21], np.arange(41))
    s = t.state()
    assert np.array_equal(r[-1, 0:9], s["d"].reshape(-1))
    assert np.array_equal(r[-1, 9:12], s["v"]) and np.array_equal(r[-1, 15:18], s["F"])
    x, y = T.build_samples(rec)
    xo, yo = M.samples(r)
    assert x.shape == (37, 34) and y.shape == (37, 6)
    # float32 rounding of double-precision inputs and targets
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-6 * max(1.0, np.abs(xo).max())
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-6 * np.abs(yo).max() + 1e-12
    # a gap in the time levels is refused
    with pytest.raises(T.TurretError):
        T.build_samples(rec[[0, 1, 2, 3, 5, 6]])


def test_linear_predictor_extrapolates_the_force_history():
    t, c = _turret(kind="oblate", seed=2)
    t.set_predictor("linear")
    t.set_log(64)
    _load(t, c)
    t.step(30)
    r = t.log_records().cpu().numpy()
    st = t.predictor_stats()
    assert st["steps"] == 30 and st["net_steps"] == 0
    F = r[:, 15:18]
    for j in range(3, 31):
        assert r[j, 29] == 0.0  # a linear prediction was made for level j
        assert np.array_equal(r[j, 23:26], 2.0 * F[j - 1] - F[j - 2])
        resid = np.linalg.norm(F[j] - r[j, 23:26]) / np.linalg.norm(F[j])
        assert abs(r[j, 22] - resid) <= 1e-12 * max(resid, 1e-300)
    assert r[0, 29] == -1.0  # no prediction for the initial level


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("bf16", 1e-4)])
def test_network_prediction_in_the_step_and_fallback(precision, tol):
    from paper_2408_15115_gb300 import turret as T
    rng = np.random.default_rng(3)
    p = I.mlp_init_params(5) * 0.3
    # outputs of order 1e-3: departures from linear extrapolation of that size
    norm = (rng.standard_normal(34) * 0.1, 0.5 + rng.random(34), rng.standard_normal(6) * 1e-3,
            1e-3 + rng.random(6) * 1e-3)
    net = T.MLP(p.astype(np.float32), batch_cap=64, precision=precision)
    net.set_norm(*[np.asarray(v, np.float32) for v in norm])
    t, c = _turret(kind="irregular", seed=4)
    t.set_predictor("mlp", net, resid_theta=1e9)  # never fall back
    t.set_log(64)
    _load(t, c)
    t.step(20)
    r = t.log_records().cpu().numpy()
    st = t.predictor_stats()
    assert st["net_steps"] == 20 - 3 and st["fallbacks"] == 3  # four history levels are needed
    pf = np.asarray(p, np.float32).astype(np.float64)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    for j in range(5, 21):
        assert r[j, 29] == 1.0
        t0 = j - 1  # the prediction for level j is made at level j - 1
        Mt = r[t0, 0:9].reshape(3, 3)
        Fh = [r[t0 - h, 15:18] for h in range(4)]
        Th = [r[t0 - h, 18:21] for h in range(4)]
        xs = (f32(M.features(Mt, r[t0, 9:12], r[t0, 12:15], Fh, Th)) - f32(norm[0])) / f32(norm[1])
        yo, _ = M.forward(pf, xs[None, :])
        yo = yo[0] * f32(norm[3]) + f32(norm[2])
        Fo, To = M.prediction(Mt, Fh, Th, yo)
        scale = np.linalg.norm(r[j, 15:18])
        assert np.abs(r[j, 23:26] - Fo).max() <= tol * scale, (j, r[j, 23:26], Fo)
    # a tiny threshold: the first network prediction misses it, every later one is linear
    t2, c2 = _turret(kind="irregular", seed=4)
    t2.set_predictor("mlp", net, resid_theta=1e-12)
    t2.set_log(64)
    _load(t2, c2)
    t2.step(20)
    made = t2.log_records().cpu().numpy()[1:, 29]
    assert list(made[:3]) == [0.0, 0.0, 0.0] and made[3] == 1.0 and np.all(made[4:] == 0.0)
    assert t2.predictor_stats()["fallback"] == 1
    net.close()


def test_relative_fallback_rule():
    # relative rule (theta = 1): a network whose outputs are all zero predicts
    # exactly the linear extrapolation, ties it and is used at every step; a
    # network with large outputs loses to it and is dropped after one step
    from paper_2408_15115_gb300 import turret as T
    zero = T.MLP(I.mlp_init_params(0).astype(np.float32) * 0.0, batch_cap=16)
    t, c = _turret(kind="oblate", seed=5)
    t.set_predictor("mlp", zero, resid_theta=1.0, relative=True)
    _load(t, c)
    t.step(30)
    st = t.predictor_stats()
    assert st["net_steps"] == 30 - 3 and st["fallbacks"] == 3
    t.close()
    p = I.mlp_init_params(1).astype(np.float32)
    p[-6:] = 50.0  # output biases: departures of 50 (standardised) from linear extrapolation
    bad = T.MLP(p, batch_cap=16)
    t, c = _turret(kind="oblate", seed=5)
    t.set_predictor("mlp", bad, resid_theta=1.0, relative=True)
    t.set_log(64)
    _load(t, c)
    t.step(30)
    made = t.log_records().cpu().numpy()[1:, 29]
    assert made[3] == 1.0 and np.all(made[4:] == 0.0)
    assert t.predictor_stats()["net_steps"] == 1
    t.close()
    zero.close()
    bad.close()


def _settle(mode, net=None, warm=False, steps=1500):
    t, c = _turret(kind="irregular", seed=7, d=12.0, re=40.0)
    if mode != "paper":
        t.set_predictor(mode, net, warm=warm, slip_eps=2e-5)
    _load(t, c)
    h = []
    for _ in range(steps // 50):
        t.step(50)
        s = t.state()
        h.append((s["F"][2], s["v"][2]))
    st = t.predictor_stats()
    t.close()
    h = np.array(h)
    return h[len(h) // 2:].mean(0), st


def test_predictor_modes_keep_the_paper_drag_and_settling():
    # predicted marker velocities (t + 1) with the paper's IBM cycles: drag and
    # settling velocity within 1 % of the paper's step
    from paper_2408_15115_gb300 import turret as T
    base, sp = _settle("paper")
    lin, _ = _settle("linear")
    net = T.MLP(I.mlp_init_params(0).astype(np.float32) * 0.0, batch_cap=16)  # outputs 0: linear extrapolation
    mlp, sm = _settle("mlp", net)
    for got in (lin, mlp):
        assert np.all(np.abs(got / base - 1.0) < 1e-2), (got, base)
    assert sm["net_steps"] > 0 and 3 * 1500 <= sp["cycles"] <= 3 * 1501  # (+ the set-up's cycles)
    # warm-started cycles carry the IBM iteration across steps: the slip left
    # after the last cycle falls well below the paper's three cold cycles
    warm, sw = _settle("linear", warm=True)
    assert max(sw["slip"][:4]) < 0.5 * max(sp["slip"][:3])
    net.close()


def test_batched_predictor_runs_equal_runs_alone():
    from paper_2408_15115_gb300 import turret as T

    def runs():
        out = []
        for k, kind in enumerate(("sphere", "prolate", "irregular")):
            t, c = _turret(kind=kind, seed=20 + k, d=10.0)
            t.set_predictor("linear", warm=(k >= 0))
            _load(t, c)
            out.append(t)
        return out
    alone = runs()
    for t in alone:
        t.step(25)
    together = runs()
    b = T.Batch(together)
    b.step(25)
    for a, t in zip(alone, together):
        sa, st = a.state(), t.state()
        for k in ("r", "v", "w", "F", "T"):
            assert np.array_equal(sa[k], st[k]), k
        assert np.array_equal(a.populations().cpu().numpy(), t.populations().cpu().numpy())
        assert a.predictor_stats()["cycles"] == t.predictor_stats()["cycles"]
    b.close()


@pytest.mark.slow
def test_trained_network_gains_over_linear_extrapolation():
    # trajectories of 48 + 8 + 8 settling runs (batched ensemble); the network
    # trained on the first 48 (early stopping on the next 8) predicts the
    # next force of the last 8 with a smaller mean error than linear
    # extrapolation 2 F(t) - F(t-1), and far better than persistence
    from paper_2408_15115_gb300 import surrogate as S
    mk = lambda n, seed: configs.ensemble(n, seed=seed, storage="f32", d_range=(8.0, 16.0))
    x, y = S.dataset(S.record_ensemble(mk(48, 11), 2000))
    xv, yv = S.dataset(S.record_ensemble(mk(8, 12), 2000))
    xt, yt = S.dataset(S.record_ensemble(mk(8, 13), 2000))
    net, hist = S.train(x, y, epochs=40, batch=4096, lr=1e-3, weight_decay=1e-4, val=(xv, yv))
    e = S.offline_errors(net, xt, yt)
    print("held-out mean relative error: network %.3e, linear %.3e, persistence %.3e" %
          (e["network"].mean(), e["linear"].mean(), e["persistence"].mean()))
    assert e["network"].mean() < e["linear"].mean()
    assert e["network"].mean() < 0.5 * e["persistence"].mean()
    net.close()


@pytest.mark.parametrize("warm,eps", [(False, 1e-4), (True, 0.0), (True, 1.0)])
def test_linear_predictor_step_vs_oracle(warm, eps):
    # the predictor option against the oracle's restatement of it: marker
    # velocities from linear extrapolation of F, T, with the paper's cold
    # cycles or warm-started ones (eps 0: all four cycles every step; eps 1:
    # one cycle per step, the slip always below it) -- the 32 x 32 x 64 closed
    # box with the seeded flow and the d = 8 sphere, 100 steps
    from oracle import oracle as O

    from cases import TOL_U_F32, gpu_velocity, make_pair, rel_max
    shape = (64, 32, 32)
    V, Tr = I.sphere(5, 8.0)
    fields = I.random_state(shape, u_amp=0.01, rho_amp=0.001, kmax=4, seed=1)
    O.set_threads(0)
    t, s = make_pair(32, 32, 64, 0.05, (1, 1, 1, 1), kappa=2.5, g=(0, 0, -1e-5), fields=fields,
                     particle=(V, Tr, (15.5, 15.5, 44.0), (0, 0, -0.01), (0.001, 0, 0)),
                     predictor=(warm, eps))
    t.step(100)
    s.step(100)
    a, b = t.state(), s.state()
    assert np.abs(a["F"] - b["F"]).max() / np.abs(b["F"]).max() < 1e-4, (a["F"], b["F"])
    assert np.abs(a["v"] - b["v"]).max() / np.abs(b["v"]).max() < 1e-5, (a["v"], b["v"])
    assert np.abs(a["w"] - b["w"]).max() / np.abs(b["w"]).max() < 1e-4, (a["w"], b["w"])
    u, _ = gpu_velocity(t)
    assert rel_max(u, s.velocity()) < TOL_U_F32
    assert t.predictor_stats()["cycles"] == s.ibm_cycles()
    t.close()
