"""Pins of the rank-model oracle (CPU): its gradient against central finite
differences, invariances of the network, and closed forms of the spectrum
summary and the rank label."""
import numpy as np

from oracle import rank_model as rm


def _params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(size=rm.NPARAM) * scale


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params(1)
    x = rng.normal(size=(7, rm.IN))
    y = rng.normal(size=7)
    loss, g = rm.loss_grad(p, x, y)
    assert np.isclose(loss, np.mean((rm.forward(p, x) - y) ** 2), rtol=1e-13)
    # every bias and output weight, and a sample of the matrix entries
    idx = np.concatenate([np.arange(rm.HID * rm.IN, rm.HID * rm.IN + rm.HID),
                          np.arange(rm.NPARAM - rm.HID - 1 - rm.HID, rm.NPARAM),
                          rng.choice(rm.HID * rm.IN, 40, replace=False),
                          rm.HID * rm.IN + rm.HID + rng.choice(rm.HID * rm.HID, 40, replace=False)])
    h = 1e-6
    for j in idx:
        e = np.zeros(rm.NPARAM)
        e[j] = h
        num = (rm.loss_grad(p + e, x, y)[0] - rm.loss_grad(p - e, x, y)[0]) / (2 * h)
        assert abs(num - g[j]) <= 1e-6 * max(1.0, abs(g[j])), (j, num, g[j])


def test_constant_network_gradient_closed_form():
    """With W2 = 0 and b2 = 0 the hidden output is 0, f = b3, so dL/db3 =
    2 mean(b3 - y) and every other gradient is 0."""
    p = _params(2)
    w1, b1, w2, b2, w3, b3 = rm.unpack(p)
    o2 = rm.HID * rm.IN + rm.HID
    p[o2:o2 + rm.HID * rm.HID + rm.HID] = 0.0
    rng = np.random.default_rng(3)
    x = rng.normal(size=(11, rm.IN))
    y = rng.normal(size=11)
    loss, g = rm.loss_grad(p, x, y)
    assert np.allclose(rm.forward(p, x), p[-1])
    assert np.isclose(g[-1], 2 * np.mean(p[-1] - y))
    assert np.isclose(loss, np.mean((p[-1] - y) ** 2))
    assert np.allclose(g[:-1], 0.0)


def test_hidden_permutation_invariance():
    p = _params(4)
    w1, b1, w2, b2, w3, b3 = rm.unpack(p)
    rng = np.random.default_rng(5)
    pi = rng.permutation(rm.HID)
    sig = rng.permutation(rm.HID)
    q = np.concatenate([w1[pi].ravel(), b1[pi], w2[sig][:, pi].ravel(), b2[sig], w3[sig], [b3]])
    x = rng.normal(size=(5, rm.IN))
    assert np.allclose(rm.forward(p, x), rm.forward(q, x), rtol=1e-12, atol=1e-12)


def test_spectrum_summary_closed_forms():
    k = 40
    flat = np.ones(k)
    assert np.allclose(rm.spectrum_summary(flat), np.log10(1.0 / k))
    # geometric weights s_mu^2 = q^mu: log10 ratio is linear in mu
    q = 0.5
    s = np.sqrt(q ** np.arange(k))
    tot = np.sum(q ** np.arange(k))
    mu = np.rint(np.arange(32) * (k - 1) / 31.0)
    assert np.allclose(rm.spectrum_summary(s), mu * np.log10(q) - np.log10(tot))
    assert np.allclose(rm.spectrum_summary(np.array([3.0])), 0.0)


def test_rank_label_closed_forms():
    assert rm.rank_label(np.ones(50)) == 50
    assert rm.rank_label(np.array([1.0, 1e-5, 1e-5])) == 1     # tail weight 2e-10
    assert rm.rank_label(np.array([1.0, 1e-2, 1e-5])) == 2     # 1e-4 then 1e-10
    s = np.sqrt(np.array([0.5, 0.25, 0.125, 0.125]))
    assert rm.rank_label(s, frac=0.74) == 2
    assert rm.rank_label(s, frac=0.76) == 3


def test_expected_records_bookkeeping():
    class R:   # stand-in for oracle.dmrg.LayerResult
        pass
    a, b = R(), R()
    a.bonds = [(1, 1), (1, 0), (2, 0), (2, 1)]
    a.spectra = [np.array([1.0, 0.5]), np.array([1.0]), np.array([0.9, 0.1]), np.array([1.0, 0.4, 0.1])]
    a.kept = [2, 1, 2, 2]
    b.bonds = [(1, 1)]
    b.spectra = [np.array([1.0, 0.3])]
    b.kept = [1]
    x, y = rm.expected_records([a, b], [[1, 4, 1], [1, 16, 1]])
    # records: (2,0) after (1,0); (2,1) after (1,1); next layer (1,1) after (2,1)
    assert x.shape == (3, rm.IN)
    assert np.allclose(x[:, 35], [1, 1, 0])
    assert np.allclose(x[:, 32], np.log2([1, 2, 2]))
    assert np.allclose(x[:, 33], np.log2([1, 4, 16]))
    assert np.allclose(x[:, 34], np.log2([2, 3, 2]))
    assert np.allclose(y, np.log2([rm.rank_label(np.array([0.9, 0.1])), rm.rank_label(np.array([1.0, 0.4])), 1]))
