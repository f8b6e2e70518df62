"""Pins of the single-site grouped oracle (oracle/single_site.py), CPU only.

Each pin is fixed by the paper or by mathematics, not by the oracle itself:
  - the group operators multiply out to the dense layer unitary;
  - the chain orders put every group of lines on consecutive sites;
  - the guess generator is SplitMix64 (published outputs);
  - at full bond dimension every layer is exact (f_delta = 1, the state equals
    the statevector), for the V, H and D groupings;
  - a layer whose gates all lie inside groups has f_delta = 1 at any chi
    (Sec. V.C: trivial layers);
  - with two groups the sweeps converge to the Eckart-Young optimum, the
    weight of the chi largest Schmidt values of the target (Sec. VI.A);
  - within a layer f never decreases, the last f equals |<new|U|old>|^2
    (Eq. fa-sup), tensors off the centre are isometries, and f_delta never
    exceeds the best-MPS bound at any group cut.
Planted mistakes in a copy of the oracle's steps must fail one of them.
"""
import numpy as np
import pytest

from oracle import dmrg as od
from oracle import mpo as om
from oracle import single_site as ss
from oracle import statevector as sv
from synthetic import circuits as sc

GROUPINGS = [("V", [1, 2, 1]), ("H", [1, 1, 1]), ("D", [2, 2, 2]), ("V", [1, 1, 1, 1])]


def _group_dense_operator(wg, sizes, order):
    """Multiply the group operators W^(tau)[w, S, T, w'] out to a dense matrix
    in qubit order (qubit 0 the most significant bit)."""
    n = sum(sizes)
    t = np.ones((1, 1, 1), dtype=np.complex128)   # [S_all, T_all, w]
    for g in wg:
        d0, ds, dt, d1 = g.shape
        t = np.einsum("xyw,wstv->xsytv", t, g).reshape(t.shape[0] * ds, t.shape[1] * dt, d1)
    t = t[:, :, 0].reshape([2] * (2 * n))          # s in site order, then t in site order
    inv = [0] * n
    for i, q in enumerate(order):
        inv[q] = i
    perm = [inv[q] for q in range(n)] + [n + inv[q] for q in range(n)]
    return t.transpose(perm).reshape(2 ** n, 2 ** n)


@pytest.mark.parametrize("kind,widths", [("V", [2, 1, 1]), ("H", [1, 2]), ("D", [2, 1, 2, 1])])
def test_group_operators_multiply_to_the_layer_unitary(kind, widths):
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 2, seed=5)
    sizes = sc.grouping(rows, cols, kind, widths)
    order = om.chain_order(rows, cols, kind)
    layer = circ.layers[0]
    wg = ss.group_mpo(om.layer_mpo(layer, order), sizes)
    u = sv.layer_unitary(rows * cols, layer)
    assert np.abs(_group_dense_operator(wg, sizes, order) - u).max() < 1e-12


def test_chain_orders_keep_groups_of_lines_contiguous():
    rows, cols = 4, 7
    for kind, line_of in (("V", lambda q: q % cols), ("H", lambda q: q // cols),
                          ("D", lambda q: q // cols + q % cols)):
        order = om.chain_order(rows, cols, kind)
        assert sorted(order) == list(range(rows * cols))
        lines = [line_of(q) for q in order]
        assert lines == sorted(lines)          # line by line along the chain
        for a, b in zip(order, order[1:]):     # consecutive sites of a line are grid neighbours
            if line_of(a) == line_of(b):
                (ra, ca), (rb, cb) = divmod(a, cols), divmod(b, cols)
                assert abs(ra - rb) + abs(ca - cb) in (1, 2)
    assert sc.grouping(4, 7, "V", [2, 3, 2]) == [8, 12, 8]
    assert sc.grouping(4, 7, "D", [3, 4, 3]) == [6, 16, 6]
    assert sum(sc.grouping(4, 7, "H", [1, 3])) == 28
    with pytest.raises(ValueError):
        sc.grouping(4, 7, "V", [2, 2])


def test_guess_generator_is_splitmix64():
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = ss.splitmix64_uniform_array(0, np.arange(3))
    assert list(u) == [(x >> 11) / 9007199254740992.0 for x in want]
    c = np.arange(0, 5000, 7)
    assert np.array_equal(ss.splitmix64_uniform_array(12345, c),
                          np.array([od.splitmix64_uniform(12345, int(k)) for k in c]))
    g = ss.random_guess([1, 3, 1], [1, 2], 9)
    assert g[0].shape == (1, 2, 3) and g[1].shape == (3, 4, 1)
    assert g[0][0, 0, 0] == complex(2 * od.splitmix64_uniform(9, 0) - 1, 2 * od.splitmix64_uniform(9, 1) - 1)
    assert g[1][0, 0, 0] == complex(2 * od.splitmix64_uniform(9, 12) - 1, 2 * od.splitmix64_uniform(9, 13) - 1)


def _run(rows, cols, kind, widths, chi, cycles=6, n_sweeps=2, seed=3):
    circ = sc.random_circuit(rows, cols, cycles, seed=seed)
    sizes = sc.grouping(rows, cols, kind, widths)
    order = om.chain_order(rows, cols, kind)
    return circ, sizes, order


@pytest.mark.parametrize("kind,widths", GROUPINGS)
def test_exact_at_full_bond_dimension(kind, widths):
    rows, cols = 3, 4
    circ, sizes, order = _run(rows, cols, kind, widths, 64)
    mps = ss.group_product_zero(sizes)
    psi = sv.zero_state(rows * cols)
    for d, layer in enumerate(circ.layers):
        wg = ss.group_mpo(om.layer_mpo(layer, order), sizes)
        mps, res, _ = ss.compress_layer(mps, wg, sizes, 64, 2, 100 + d)
        psi = sv.apply_layer(psi, layer)
        assert abs(res.f_delta - 1) < 1e-12
        # one sweep from the random guess already reaches the exact state
        assert abs(res.f[len(sizes) - 1] - 1) < 1e-12
    dense = ss.group_dense(mps, sizes, order)
    assert abs(abs(np.vdot(dense.reshape(-1), psi.reshape(-1))) - 1) < 1e-12


def test_trivial_layers_are_lossless():
    """Vertical gates (patterns B, D) lie inside column groups: a layer of
    only those keeps f_delta = 1 whatever chi (Sec. V.C)."""
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 6, seed=11)
    sizes = sc.grouping(rows, cols, "V", [1, 1, 1, 1])
    order = om.chain_order(rows, cols, "V")
    mps = ss.group_product_zero(sizes)
    chi = 3
    for d, layer in enumerate(circ.layers[:2]):
        mps, res, _ = ss.compress_layer(mps, ss.group_mpo(om.layer_mpo(layer, order), sizes),
                                        sizes, chi, 2, 7 + d)
    assert res.f_delta < 0.999   # the state is truncated
    edges = sc.grid_edges(rows, cols)
    vertical = edges["B"] + edges["D"]
    rng = np.random.default_rng(4)
    trivial = [(q, -1, sc.sqrt_pauli("XYW"[rng.integers(3)])) for q in range(rows * cols)]
    trivial += [(a, b, sc.fsim(np.pi / 2, np.pi / 6)) for (a, b) in vertical]
    wg = ss.group_mpo(om.layer_mpo(trivial, order), sizes)
    assert all(g.shape[3] == 1 for g in wg)     # no operator bond between groups
    mps2, res2, _ = ss.compress_layer(mps, wg, sizes, chi, 2, 99)
    assert abs(res2.f_delta - 1) < 1e-12


def test_two_groups_reach_eckart_young():
    """m = 2: alternating updates are a subspace iteration on the one bond;
    they converge to the chi leading Schmidt vectors of U|Psi_Q>, whose weight
    is the best possible f (Sec. VI.A)."""
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 4, seed=2)
    sizes = sc.grouping(rows, cols, "V", [2, 2])
    order = om.chain_order(rows, cols, "V")
    mps = ss.group_product_zero(sizes)
    mps, _, _ = ss.compress_layer(mps, ss.group_mpo(om.layer_mpo(circ.layers[0], order), sizes),
                                  sizes, 64, 2, 1)
    old = ss.group_dense(mps, sizes, order)
    layer = circ.layers[1]
    target = sv.apply_layer(old, layer)
    s = sv.schmidt_values(target, order[:sizes[0]])
    # the cut with the widest gap among chi = 3..10: the iteration converges
    # as (s_{chi+1} / s_chi)^(2 n_sweeps)
    chi = max(range(3, 11), key=lambda k: s[k - 1] / s[k])
    assert (s[chi] / s[chi - 1]) ** 2 < 0.8
    best = float(np.sum(s[:chi] ** 2))
    _, res, _ = ss.compress_layer(mps, ss.group_mpo(om.layer_mpo(layer, order), sizes), sizes, chi, 200, 5)
    assert res.f_delta <= best + 1e-12
    assert best - res.f_delta < 1e-9, (best, res.f_delta, s[chi - 1:chi + 1])


@pytest.mark.parametrize("kind,widths", GROUPINGS)
def test_step_invariants(kind, widths):
    rows, cols = 3, 4
    circ, sizes, order = _run(rows, cols, kind, widths, 4, cycles=6, seed=8)
    chi = 4
    mps = ss.group_product_zero(sizes)
    for d, layer in enumerate(circ.layers):
        old = ss.group_dense(mps, sizes, order)
        wg = ss.group_mpo(om.layer_mpo(layer, order), sizes)
        new, res, centre = ss.compress_layer(mps, wg, sizes, chi, 3, 40 + d)
        h = np.array(res.f)
        assert np.all(np.diff(h) >= -1e-12)
        target = sv.apply_layer(old, layer)
        dense = ss.group_dense(new, sizes, order)
        assert abs(abs(np.vdot(dense.reshape(-1), target.reshape(-1))) ** 2 - res.f_delta) < 1e-12
        assert abs(np.linalg.norm(dense) - 1) < 1e-12
        for tau, a in enumerate(new):
            al, s, ar = a.shape
            if tau < centre:
                m = a.reshape(al * s, ar)
                assert np.abs(m.conj().T @ m - np.eye(ar)).max() < 1e-12
            elif tau > centre:
                m = a.reshape(al, s * ar)
                assert np.abs(m @ m.conj().T - np.eye(al)).max() < 1e-12
        left = 0
        for r in sizes[:-1]:
            left += r
            sch = sv.schmidt_values(target, order[:left])
            assert res.f_delta <= float(np.sum(sch[:chi] ** 2)) + 1e-12
        mps = new


def _exact_error():
    """Largest departure from what an exact run guarantees: the final overlap
    with the statevector, every f of every layer equal to 1 from the end of
    the first sweep on (the update count of one sweep is m), f <= 1."""
    rows, cols = 3, 4
    circ = sc.random_circuit(rows, cols, 4, seed=3)
    sizes = sc.grouping(rows, cols, "V", [1, 2, 1])
    order = om.chain_order(rows, cols, "V")
    mpos = [om.layer_mpo(l, order) for l in circ.layers]
    mps, results, _ = ss.run_circuit(mpos, sizes, 64, 2, 5)
    exact = sv.run(rows * cols, circ.layers)[-1]
    dense = ss.group_dense(mps, sizes, order)
    err = 1 - abs(np.vdot(dense.reshape(-1), exact.reshape(-1)))
    for r in results:
        f = np.array(r.f[len(sizes) - 1:])
        err = max(err, np.abs(f - 1).max())
    return err


def test_unpatched_single_site_oracle_is_exact():
    assert _exact_error() < 1e-12


@pytest.mark.parametrize("bug", ["operator_transposed", "env_no_conj", "y_wrong_leg", "right_env_no_conj",
                                 "group_bits_swapped"])
def test_planted_bug_is_caught(monkeypatch, bug):
    if bug == "operator_transposed":
        orig = ss.x_of
        monkeypatch.setattr(ss, "x_of", lambda l, b, w: orig(l, b, w.transpose(0, 2, 1, 3)))
    elif bug == "env_no_conj":
        monkeypatch.setattr(ss, "env_left", lambda a, x: np.einsum("ask,aswb->kwb", a, x))
    elif bug == "y_wrong_leg":
        orig = ss.y_of
        monkeypatch.setattr(ss, "y_of", lambda r, b, w: orig(r, b, w.transpose(0, 2, 1, 3)))
    elif bug == "right_env_no_conj":
        monkeypatch.setattr(ss, "env_right", lambda a, y: np.einsum("ksc,scwb->kwb", a, y))
    elif bug == "group_bits_swapped":
        orig = ss.group_mpo

        def swapped(w, sizes):
            out = orig(w, sizes)
            res = []
            for g, r in zip(out, sizes):
                if r >= 2:
                    d0, ds, dt, d1 = g.shape
                    g = g.reshape(d0, 2, ds // 2, dt, d1).transpose(0, 2, 1, 3, 4).reshape(d0, ds, dt, d1)
                res.append(g)
            return res
        monkeypatch.setattr(ss, "group_mpo", swapped)
    assert _exact_error() > 1e-3
