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
