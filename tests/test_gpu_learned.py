"""The count predictor (feast_mlp_*) against the FP64 oracle, and what the
trained network gains over the plain stochastic count when choosing m0."""
import numpy as np
import pytest

import workloads
from helpers import lib
from oracle import brute, mlp as omlp

pytestmark = pytest.mark.gpu


def _net(fg, d_in, width, seed, B):
    rng = np.random.default_rng(seed)
    p = workloads.mlp_init(d_in, width, seed)
    X = rng.standard_normal((B, d_in)).astype(np.float32)
    y = rng.standard_normal(B).astype(np.float32)
    mean, scale = X.mean(0), X.std(0) + 0.5
    return fg.MLP(d_in, width, 256, p, mean, scale), p, X, y, mean, scale


@pytest.mark.parametrize("width", [16, 256])
def test_forward_and_gradient_match_oracle(width):
    fg = lib()
    d_in, B = 17, 96
    net, p, X, y, mean, scale = _net(fg, d_in, width, 3, B)
    out = net.predict(X)
    ref, _ = omlp.forward(p, X, mean, scale, d_in, width)
    assert np.max(np.abs(out - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    loss, g = net.grad(X, y)
    lref, gref = omlp.loss_and_grad(p, X, y, mean, scale, d_in, width)
    assert abs(loss - lref) <= 1e-4 * lref
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_adam_steps_match_oracle():
    fg = lib()
    d_in, width, B = 17, 32, 64
    net, p, X, y, mean, scale = _net(fg, d_in, width, 4, B)
    batches = workloads.batch_schedule(B, 32, 3, seed=1)
    net.train(X, y, batches, lr=1e-2)
    pr, m, v = p.astype(np.float64), 0.0, 0.0
    for t, bidx in enumerate(batches, start=1):
        _, g = omlp.loss_and_grad(pr, X[bidx], y[bidx], mean, scale, d_in, width)
        pr, m, v = omlp.adam_step(pr, g, m, v, t, 1e-2)
    got = net.params()
    # Adam divides by sqrt(v): entries whose gradient is at rounding level can
    # move by up to lr with either sign, so compare the update as a whole and
    # require almost every entry to agree closely
    upd = pr - p
    assert np.linalg.norm(got - pr) <= 2e-2 * np.linalg.norm(upd)
    assert np.mean(np.abs(got - pr) > 1e-4) < 0.01


def test_learned_m0_beats_plain_stochastic_count():
    """Config-5 style family at n = 256: the network trained on (p, moments) ->
    count pairs generated by the method predicts the count better than the plain
    stochastic trace estimate Re mu_0, and the m0 it implies is never smaller
    than the true count on the held-out draws."""
    fg = lib()
    from paper_1404_2891_gb300 import learned_m0 as lm
    fam = workloads.parametric_family(n=256, seed=5, n_train=240, n_test=60)
    n = 256
    feats, labels = [], []
    for i, p in enumerate(np.concatenate([fam["p_train"], fam["p_test"]])):
        feats.append(lm.features(fam, p, workloads.rademacher(n, 32, 1000 + i)))
        labels.append(lm.label(fam, p, workloads.random_block(n, 96, 5000 + i)))
    feats = np.array(feats)
    labels = np.array([np.nan if l is None else l for l in labels], dtype=float)
    assert np.isfinite(labels).all()
    # the method's counts agree with brute force on a sample of the family
    for i in (0, 7, 250):
        p = np.concatenate([fam["p_train"], fam["p_test"]])[i]
        c = fam["contour"]
        assert labels[i] == len(brute.inside_spectrum(fam["A0"] + p * fam["A1"], None, c["c"], c["R"], c["a"]))
    ntr = len(fam["p_train"])
    Xtr, ytr, Xte, yte = feats[:ntr], labels[:ntr], feats[ntr:], labels[ntr:]
    pred_model = lm.CountPredictor(Xtr, width=256, init_params=workloads.mlp_init(lm.D_IN, 256, 11))
    pred_model.fit(Xtr, ytr, workloads.batch_schedule(ntr, 48, 1500, seed=12), lr=1e-3)
    pred = pred_model.predict(Xte)
    plain = Xte[:, 1]  # Re mu_0
    mae_net = np.mean(np.abs(pred - yte))
    mae_plain = np.mean(np.abs(plain - yte))
    assert mae_net < mae_plain, (mae_net, mae_plain)
    m0_net = np.array([lm.m0_rule(v) for v in pred])
    assert np.all(m0_net >= yte)
