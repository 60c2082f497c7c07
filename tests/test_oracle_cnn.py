"""Pins of the warm-start network oracle (oracle/cnn.py) against things other
than itself: a library cross-correlation, finite differences of its own loss
(brute force on a tiny grid), the closed form of Adam's first step, exact
bfloat16 values, and the linearity of Eq. (8) through the training pairs."""
import numpy as np
import pytest
from scipy import signal

import oracle
from oracle import cnn
import synthetic


def test_conv_is_the_library_cross_correlation():
    rng = np.random.default_rng(0)
    B, H, W, ci, co = 2, 7, 11, 3, 4
    h = rng.standard_normal((B, H, W, ci))
    Wt = rng.standard_normal((9, co, ci))
    b = rng.standard_normal(co)
    a = cnn.conv(h, Wt, b)
    for bb in range(B):
        for o in range(co):
            ref = np.full((H, W), b[o])
            for c in range(ci):
                k = Wt[:, o, c].reshape(3, 3)       # k[dy + 1, dx + 1]
                ref += signal.correlate2d(h[bb, :, :, c], k, mode="same", boundary="fill")
            assert np.allclose(a[bb, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_parameter_count_and_layout():
    assert cnn.n_params() == (9 * 32 + 32) + 4 * (9 * 32 * 32 + 32) + (9 * 32 + 1)
    p = np.arange(cnn.n_params(), dtype=np.float64)
    assert np.array_equal(cnn.pack(cnn.unpack(p)), p)
    (W1, b1) = cnn.unpack(p)[0]
    assert W1.shape == (9, 32, 1) and b1[0] == 9 * 32


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    B, H, W = 2, 5, 6
    x = rng.standard_normal((B, H, W))
    t = rng.standard_normal((B, H, W))
    p = cnn.init_params(3)
    p[cnn.n_params() - 1] = 0.3
    L, g = cnn.loss_and_grad(p, x, t)
    assert L == pytest.approx(cnn.loss(p, x, t), rel=1e-14)
    # every bias and a spread of weights of every layer
    idx, o = [], 0
    for nw, nb in cnn.layer_sizes():
        idx += list(rng.choice(nw, size=min(nw, 40), replace=False) + o)
        idx += list(range(o + nw, o + nw + nb))
        o += nw + nb
    h = 1e-6
    bad = 0
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (cnn.loss(pp, x, t) - cnn.loss(pm, x, t)) / (2 * h)
        if abs(fd - g[k]) > 1e-6 * abs(g).max() + 1e-4 * abs(g[k]):
            bad += 1                       # a ReLU kink inside [-h, h]
    assert bad <= 0.02 * len(idx)


def test_gradient_check_catches_a_wrong_tap():
    """The finite-difference pin fails for a plausible mistake: the back
    propagation using the un-mirrored tap."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 6))
    t = rng.standard_normal((1, 5, 6))
    p = cnn.init_params(4)
    _, g = cnn.loss_and_grad(p, x, t)
    saved = cnn.TAPS[:]
    try:
        cnn.TAPS[:] = saved[::-1]          # a transposed stencil in both passes
        _, gw = cnn.loss_and_grad(p, x, t)
    finally:
        cnn.TAPS[:] = saved
    assert np.abs(gw - g).max() > 1e-3 * np.abs(g).max()


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    w1, m, v = cnn.adam_step(w, g, z, z, 1, lr=1e-2, eps=1e-8)
    assert np.allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps moving each weight by lr (bias correction)
    w2, _, _ = cnn.adam_step(w1, g, m, v, 2, lr=1e-2, eps=0.0)
    assert np.allclose(w2, w1 - 1e-2 * np.sign(g), rtol=1e-12)


def test_bf16_rounding_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 3.0e38, 1e-40])
    r = cnn.round_bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                              # tie to even (down)
    assert r[2] == 1.0 + 2.0 ** -6                  # tie to even (up)
    assert r[3] == 1.0 + 2.0 ** -7                  # representable
    assert r[4] == -2.5
    assert np.isfinite(r[5]) or np.isinf(r[5])
    x = np.random.default_rng(6).standard_normal(1000)
    assert np.all(np.abs(cnn.round_bf16(x) - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-12))   # half an ulp (8-bit significand)


def test_bf16_mirror_is_close_to_exact():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((1, 9, 8))
    t = rng.standard_normal((1, 9, 8))
    p = cnn.init_params(8)
    L, g = cnn.loss_and_grad(p, x, t)
    Lb, gb = cnn.loss_and_grad(p, x, t, bf16=True)
    assert abs(Lb - L) <= 0.05 * L
    assert np.linalg.norm(gb - g) <= 0.05 * np.linalg.norm(g)


def _solved(cfg, xs, parts=None, V=None):
    c = dict(cfg)
    if V is not None:
        c["V0"] = V
    o = oracle.Oracle(c, fp64=True)
    o.set_cross_sections(xs)
    if parts is not None:
        o.load(parts)
    o.prime()
    n = c["nz"] + 1
    rho = cnn.node_density(sum(o.rho()).astype(np.float64), c["weight"], c["dz"], c["dr"], c["nz"], c["nr"])
    return rho, o.phi().reshape(n, -1)


def test_training_pairs_follow_eq8_linearity(xs):
    """Through the oracle's Poisson solve: a charge-free gap gives t = 0, the
    target is invariant to scaling the charge, the warm start built from the
    exact target reproduces the potential, and the delta pair of two states
    equals the absolute pair of their charge difference."""
    cfg, parts = synthetic.rz_plume(n=16, total=6e3, seed=9)
    cfg.update(field_on=1, inject_on=0, poisson_tol=1e-13, oracle_poisson_tol=1e-13)
    n = cfg["nz"] + 1
    dz, V = cfg["dz"], cfg["V0"]
    rho, phi = _solved(cfg, xs, parts)
    # the volumes sum to the cylinder: a uniform density is returned as given
    vol = 1.602176634e-19 * cfg["weight"] / 2.0 ** 32 / cnn.node_density(np.ones(rho.size), cfg["weight"], dz,
                                                                       cfg["dr"], cfg["nz"], cfg["nr"])
    assert vol.sum() == pytest.approx(np.pi * (cfg["nr"] * cfg["dr"]) ** 2 * cfg["nz"] * dz, rel=1e-12)
    x, t = cnn.training_pair(rho, phi, V, dz)
    assert np.abs(x).max() == pytest.approx(1.0)
    assert np.abs(t).max() > 0
    zV = V * np.arange(n)[:, None] / (n - 1)
    x2, t2 = cnn.training_pair(3.0 * rho, zV + 3.0 * (phi - zV), V, dz)
    assert np.allclose(x2, x) and np.allclose(t2, t, rtol=1e-12, atol=1e-15)
    phi0 = cnn.warm_start(t, np.abs(rho).max(), V, dz)
    assert np.allclose(phi0, phi, rtol=1e-12, atol=1e-9 * V)
    _, tz = cnn.training_pair(np.zeros_like(rho), phi, V, dz)
    assert not tz.any()
    rho0, phiL = _solved(cfg, xs)
    assert not rho0.any()
    _, tl = cnn.training_pair(rho, phiL, V, dz)
    assert np.abs(tl).max() <= 1e-9 * np.abs(t).max()
    # a second state: half of the particles, another voltage
    half = {k: v[::2] for k, v in parts.items()}
    rho_b, phi_b = _solved(cfg, xs, half, V=1.7e3)
    xd, td = cnn.training_pair(rho, phi, V, dz, rho_prev=rho_b, phi_prev=phi_b, V_prev=1.7e3)
    # the charge difference is the other half of the particles (integer
    # deposits add exactly); solved alone with the anode grounded it gives,
    # by the linearity of Eq. (8), the same pair
    odd = {k: v[1::2] for k, v in parts.items()}
    rho_o, phi_o = _solved(cfg, xs, odd, V=0.0)
    m = np.abs(rho - rho_b).max()
    assert np.allclose(rho - rho_b, rho_o, rtol=1e-12, atol=1e-12 * m)
    xa, ta = cnn.training_pair(rho_o, phi_o, 0.0, dz)
    assert np.allclose(xd, xa, rtol=1e-10, atol=1e-12)
    assert np.allclose(td, ta, rtol=1e-7, atol=1e-7 * np.abs(ta).max())
    assert np.allclose(cnn.warm_start(td, m, V, dz, phi_prev=phi_b, V_prev=1.7e3), phi, rtol=1e-12, atol=1e-9 * V)


def test_rz_operator_is_the_solvers_finite_volume_equation(xs):
    """Through the oracle's own Poisson solve (conjugate gradients on its
    finite-volume equations): the target t of a pair satisfies S t = w x on
    the interior rows, to the solve's tolerance; S is symmetric.  Planted
    mistakes (Verboncoeur's 1/6 for the axis volume, a face past the outer
    radius) break the identity."""
    cfg, parts = synthetic.rz_plume(n=16, total=6e3, seed=9)
    cfg.update(field_on=1, inject_on=0, poisson_tol=1e-13, oracle_poisson_tol=1e-13)
    rho, phi = _solved(cfg, xs, parts)
    x, t = cnn.training_pair(rho, phi, cfg["V0"], cfg["dz"])
    _, _, w = cnn.rz_weights(x.shape[1])
    scale = np.abs(w * x).max()
    r = cnn.rz_residual(x, t)
    assert np.abs(r).max() <= 1e-9 * scale
    # symmetric on the interior rows
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2,) + t.shape)
    a[[0, -1]] = 0.0
    b[[0, -1]] = 0.0
    assert np.vdot(a, cnn.rz_operator(b)) == pytest.approx(np.vdot(cnn.rz_operator(a), b), rel=1e-12)
    saved = cnn.rz_weights

    def axis_sixth(W):
        ap, am, w_ = saved(W)
        w_ = w_.copy()
        w_[0] = 1.0 / 6.0
        return ap, am, w_

    def outer_face(W):
        ap, am, w_ = saved(W)
        ap = ap.copy()
        ap[-1] = W - 0.5
        return ap, am, w_

    for bad in (axis_sixth, outer_face):
        cnn.rz_weights = bad
        try:
            assert np.abs(cnn.rz_residual(x, t)).max() > 1e-6 * scale, bad.__name__
        finally:
            cnn.rz_weights = saved


def test_extrapolated_pair_is_the_pair_of_the_second_difference(xs):
    """Linearity of Eq. (8): the extrapolated pair of three states equals the
    absolute pair of rho - 2 rho' + rho'' solved with the anode at
    V - 2 V' + V''; with states linear in time (rho'' , rho', rho equally
    spaced) x and t vanish."""
    cfg, parts = synthetic.rz_plume(n=16, total=6e3, seed=9)
    cfg.update(field_on=1, inject_on=0, poisson_tol=1e-13, oracle_poisson_tol=1e-13)
    dz = cfg["dz"]
    thirds = [{k: v[q::3] for k, v in parts.items()} for q in range(3)]
    two = {k: np.concatenate([thirds[0][k], thirds[1][k]]) for k in parts}
    # states: rho2 = A (V 1.5 kV), rho1 = A + B (2.1 kV), rho = all (2.9 kV)
    s2 = _solved(cfg, xs, thirds[0], V=1.5e3)
    s1 = _solved(cfg, xs, two, V=2.1e3)
    s0 = _solved(cfg, xs, parts, V=2.9e3)
    x, t = cnn.training_pair_extrap(s0[0], s0[1], 2.9e3, dz, s1[0], s1[1], 2.1e3, s2[0], s2[1], 1.5e3)
    # rho - 2 rho1 + rho2 = C - B (integer deposits add exactly): solved with
    # V - 2 V1 + V2 = 0.2 kV it gives the same pair
    sB = _solved(cfg, xs, thirds[1], V=0.0)
    sC = _solved(cfg, xs, thirds[2], V=0.2e3)
    d = s0[0] - 2.0 * s1[0] + s2[0]
    assert np.allclose(d, sC[0] - sB[0], rtol=1e-12, atol=1e-12 * np.abs(d).max())
    xa, ta = cnn.training_pair(sC[0] - sB[0], sC[1] - sB[1], 0.2e3, dz)
    assert np.allclose(x, xa, rtol=1e-10, atol=1e-12)
    assert np.allclose(t, ta, rtol=1e-7, atol=1e-7 * np.abs(ta).max())
    # the exact target leaves no residual
    _, _, w = cnn.rz_weights(x.shape[1])
    assert np.abs(cnn.rz_residual(x, t)).max() <= 1e-9 * np.abs(w * x).max()
    # equally spaced states: nothing for the network to add
    x0, t0 = cnn.training_pair_extrap(s0[0], s0[1], 2.9e3, dz, s0[0], s0[1], 2.9e3, s0[0], s0[1], 2.9e3)
    assert not x0.any() and not t0.any()


def test_residual_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    B, H, W = 2, 6, 7
    x = rng.standard_normal((B, H, W))
    p = cnn.init_params(6)
    p[cnn.n_params() - 1] = 0.2
    L, g = cnn.resid_loss_and_grad(p, x)
    y, _ = cnn.forward(p, x)
    r = cnn.rz_residual(x, y)
    assert L == pytest.approx((r * r).sum() / (B * (H - 2) * W), rel=1e-14)
    idx, o = [], 0
    for nw, nb in cnn.layer_sizes():
        idx += list(rng.choice(nw, size=min(nw, 30), replace=False) + o)
        idx += list(range(o + nw, o + nw + nb))
        o += nw + nb

    def loss_of(q):
        yq, _ = cnn.forward(q, x)
        rq = cnn.rz_residual(x, yq)
        return (rq * rq).sum() / (B * (H - 2) * W)

    h = 1e-6
    bad = 0
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (loss_of(pp) - loss_of(pm)) / (2 * h)
        if abs(fd - g[k]) > 1e-6 * abs(g).max() + 1e-4 * abs(g[k]):
            bad += 1                       # a ReLU kink inside [-h, h]
    assert bad <= 0.02 * len(idx)
