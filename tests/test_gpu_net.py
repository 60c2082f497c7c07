"""The warm-start network on the GPU against the float64 oracle (oracle/cnn.py,
in its bfloat16 mirror): forward pass, loss, every parameter's gradient and
Adam; the training pairs of a simulation against the oracle's; and the
Poisson warm-start modes (the solve still reaches its tolerance from any
starting point).

Tolerances: both sides round the same values to bfloat16 and differ in the
order of their float sums (about 1e-6 relative), which now and then moves a
value across a bfloat16 rounding boundary (one unit in the 8th bit).  Such
flips stay rare and isolated, so the norms agree to ~1e-4; the bounds below
leave a factor of ten or more."""
import numpy as np
import pytest

import oracle
from oracle import cnn
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def pd(torch):
    import paper_2109_00214_gb300 as m
    m.load_library()
    return m


def _params(seed):
    p = cnn.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    o = 0
    for nw, nb in cnn.layer_sizes():
        p[o + nw:o + nw + nb] = 0.05 * rng.standard_normal(nb)
        o += nw + nb
    return p.astype(np.float32)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("B,H,W", [(2, 21, 37), (1, 8, 16), (3, 5, 3)])
def test_forward_loss_and_gradients_match_the_oracle(pd, torch, B, H, W):
    rng = np.random.default_rng(B * 1000 + H * 10 + W)
    p = _params(B + H + W)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = (0.1 * rng.standard_normal((B, H, W))).astype(np.float32)
    net = pd.Net(B * H * W, params=p)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    y = net.forward(xd).cpu().numpy()
    p64 = p.astype(np.float64)
    yo, _ = cnn.forward(p64, x, bf16=True)
    assert _rel(y, yo) <= 2e-3
    loss, g = net.loss_grad(xd, td, want_grads=True)
    lo, go = cnn.loss_and_grad(p64, x, t, bf16=True)
    assert loss == pytest.approx(lo, rel=2e-3)
    o = 0
    for l, (nw, nb) in enumerate(cnn.layer_sizes()):
        assert _rel(g[o:o + nw], go[o:o + nw]) <= 1e-2, ("weights", l)
        assert _rel(g[o + nw:o + nw + nb], go[o + nw:o + nw + nb]) <= 1e-2, ("biases", l)
        o += nw + nb
    net.close()


def test_gradient_check_fails_for_a_wrong_gradient(pd, torch):
    """The comparison above has teeth: the GPU gradient is far from the
    oracle's gradient of a perturbed problem (targets shifted)."""
    rng = np.random.default_rng(3)
    B, H, W = 1, 12, 20
    p = _params(5)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = (0.1 * rng.standard_normal((B, H, W))).astype(np.float32)
    net = pd.Net(B * H * W, params=p)
    _, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), want_grads=True)
    _, go = cnn.loss_and_grad(p.astype(np.float64), x, t + 0.05, bf16=True)
    assert _rel(g, go) > 0.05
    net.close()


def test_adam_matches_the_oracle(pd, torch):
    rng = np.random.default_rng(4)
    B, H, W = 2, 10, 18
    p = _params(6)
    net = pd.Net(B * H * W, params=p)
    w = p.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for k in (1, 2, 3):
        x = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
        t = torch.from_numpy((0.1 * rng.standard_normal((B, H, W))).astype(np.float32)).cuda()
        _, g = net.loss_grad(x, t, want_grads=True)
        net.adam(lr=1e-3)
        w, m, v = cnn.adam_step(w, g.astype(np.float64), m, v, k, lr=1e-3)
        assert np.abs(net.params() - w).max() <= 1e-6
    net.close()


def test_training_lowers_the_loss(pd, torch):
    rng = np.random.default_rng(8)
    B, H, W = 4, 33, 33
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    x = np.stack([np.exp(-((ii - rng.uniform(5, 28)) ** 2 + (jj - rng.uniform(5, 28)) ** 2) / 20.0)
                  for _ in range(B)]).astype(np.float32)
    t = (0.3 * x + 0.1 * np.roll(x, 2, axis=1)).astype(np.float32)
    net = pd.Net(B * H * W, params=_params(9))
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0, _ = net.loss_grad(xd, td)
    for _ in range(150):
        net.loss_grad(xd, td, want_grads=False)
        net.adam(lr=2e-3)
    l1, _ = net.loss_grad(xd, td)
    assert l1 < 0.2 * l0
    net.close()


def _plume(n=32, total=2e4, seed=21):
    cfg, parts = synthetic.rz_plume(n=n, total=total, seed=seed)
    cfg.update(field_on=1, inject_on=0, poisson_tol=1e-10, oracle_poisson_tol=1e-12)
    return cfg, parts


def test_training_pairs_match_the_oracle(pd, torch, xs):
    cfg, parts = _plume()
    sim = pd.Simulation(cfg, xs)
    sim.load(parts)
    sim.step(0)
    x, t = (a.cpu().numpy().astype(np.float64).reshape(sim.nzn, sim.nrn) for a in sim.warmstart_pairs())
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    rho = cnn.node_density(sum(o.rho()), cfg["weight"], cfg["dz"], cfg["dr"], cfg["nz"], cfg["nr"])
    xo, to = cnn.training_pair(rho, o.phi().reshape(sim.nzn, sim.nrn), cfg["V0"], cfg["dz"])
    assert np.abs(x - xo).max() <= 1e-6
    assert np.abs(t - to).max() <= 1e-5 * np.abs(to).max()
    assert np.abs(to).max() > 0


def test_delta_pairs_match_the_oracle(pd, torch, xs):
    """Pairs of two consecutive solves (load + solve, one step + solve).  One
    step moves the particles identically on both sides (the two potentials
    differ by far less than a float rounding of the push), so the charge is
    bit-identical and the potentials agree to the solve tolerance."""
    cfg, parts = _plume()
    cfg.update(poisson_tol=1e-12, oracle_poisson_tol=1e-13)
    # a quarter of the load in the row at the anode: the charge it absorbs in
    # the step drives the circuit, so the anode voltage of the two solves differs
    parts = {k: v.copy() for k, v in parts.items()}
    parts["iz"][::4] = cfg["nz"] - 1
    sim = pd.Simulation(cfg, xs)
    sim.load(parts)
    sim.step(0)
    with pytest.raises(pd.PdError):
        sim.warmstart_pairs("delta")          # one solve only
    sim.step(1)
    x, t = (a.cpu().numpy().astype(np.float64).reshape(sim.nzn, sim.nrn) for a in sim.warmstart_pairs("delta"))
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    grid = (cfg["weight"], cfg["dz"], cfg["dr"], cfg["nz"], cfg["nr"])
    rho1, phi1, V1 = cnn.node_density(sum(o.rho()), *grid), o.phi().reshape(sim.nzn, sim.nrn), cfg["V0"]
    o.step(1)
    rho2, phi2, V2 = cnn.node_density(sum(o.rho()), *grid), o.phi().reshape(sim.nzn, sim.nrn), o.scalars()["V"]
    assert V2 != V1
    xo, to = cnn.training_pair(rho2, phi2, V2, cfg["dz"], rho_prev=rho1, phi_prev=phi1, V_prev=V1)
    assert np.abs(xo).max() == pytest.approx(1.0)
    assert np.abs(x - xo).max() <= 1e-6
    assert np.abs(t - to).max() <= 1e-3 * np.abs(to).max()


def test_warm_start_modes_reach_the_tolerance(pd, torch, xs):
    cfg, parts = _plume(n=64, total=6e4)
    net = pd.Net((cfg["nz"] + 1) * (cfg["nr"] + 1), params=_params(10))
    cycles = {}
    for mode in ("previous", "cold", "learned", "learned_delta", "learned_extrap"):
        sim = pd.Simulation(cfg, xs)
        sim.load(parts)
        sim.step(2)
        sim.set_warm_start(mode, net if mode.startswith("learned") else None)
        sim.step(1)
        sc = sim.scalars()
        assert sc["poisson_relres"] <= cfg["poisson_tol"], mode
        cycles[mode] = sc["poisson_cycles"]
        sim.close()
    assert cycles["cold"] >= cycles["previous"]
    net.close()


@pytest.mark.parametrize("B,H,W", [(2, 21, 37), (1, 8, 16), (3, 5, 3)])
def test_residual_loss_and_gradients_match_the_oracle(pd, torch, B, H, W):
    rng = np.random.default_rng(7 * B + H + W)
    p = _params(3 * B + W)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    net = pd.Net(B * H * W, params=p)
    loss, g = net.loss_grad_rz(torch.from_numpy(x).cuda(), want_grads=True)
    lo, go = cnn.resid_loss_and_grad(p.astype(np.float64), x, bf16=True)
    assert loss == pytest.approx(lo, rel=2e-3)
    o = 0
    for l, (nw, nb) in enumerate(cnn.layer_sizes()):
        assert _rel(g[o:o + nw], go[o:o + nw]) <= 1e-2, ("weights", l)
        assert _rel(g[o + nw:o + nw + nb], go[o + nw:o + nw + nb]) <= 1e-2, ("biases", l)
        o += nw + nb
    net.close()


def test_extrapolated_pairs_match_the_oracle(pd, torch, xs):
    """Pairs of three consecutive solves (load + solve, two steps with a
    solve each) against the oracle's definition on the oracle's own states:
    the float oracle moves the particles as the library does, so the charge
    is bit-identical and the potentials agree to the solve tolerance."""
    cfg, parts = _plume()
    cfg.update(poisson_tol=1e-12, oracle_poisson_tol=1e-13)
    parts = {k: v.copy() for k, v in parts.items()}
    parts["iz"][::4] = cfg["nz"] - 1
    sim = pd.Simulation(cfg, xs)
    sim.load(parts)
    sim.step(1)
    with pytest.raises(pd.PdError):
        sim.warmstart_pairs("extrap")         # two solves only
    sim.step(1)
    x, t = (a.cpu().numpy().astype(np.float64).reshape(sim.nzn, sim.nrn) for a in sim.warmstart_pairs("extrap"))
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    grid = (cfg["weight"], cfg["dz"], cfg["dr"], cfg["nz"], cfg["nr"])
    st = []
    for k in range(3):
        if k:
            o.step(1)
        st.append((cnn.node_density(sum(o.rho()), *grid), o.phi().reshape(sim.nzn, sim.nrn), o.scalars()["V"]))
    (r2, p2, V2), (r1, p1, V1), (r0, p0, V0) = st
    xo, to = cnn.training_pair_extrap(r0, p0, V0, cfg["dz"], r1, p1, V1, r2, p2, V2)
    assert np.abs(xo).max() == pytest.approx(1.0)
    assert np.abs(x - xo).max() <= 1e-6
    assert np.abs(t - to).max() <= 1e-3 * np.abs(to).max()


def test_learned_correction_beats_the_extrapolated_start(pd, torch, xs):
    """The network trained on the residual its correction leaves (three
    training runs, 128^2 r-z plume) starts the solves of a held-out run
    closer than the potential extrapolated in time: a smaller starting
    residual and no more multigrid cycles to 1e-8."""
    from paper_2109_00214_gb300 import warmstart as W
    n = 128
    runs = []
    for k in range(4):
        cfg, parts = synthetic.rz_plume(n=n, total=2.5e5, seed=300 + k)
        cfg.update(field_on=1, inject_on=0, run=k, V0=1e3 * (2 + 2 * k), poisson_tol=1e-8)
        runs.append((cfg, parts))
    train_runs, test_run = runs[:3], runs[3]
    pairs = W.collect_pairs([c for c, _ in train_runs], [p for _, p in train_runs], xs, 60, kinds=("extrap",))
    X = pairs["extrap"][0].flatten(0, 1)
    net = pd.Net(8 * (n + 1) ** 2, params=cnn.init_params(5).astype(np.float32))
    W.train(net, [(X, X)], 2000, 8, lr=3e-3, lr_final=5e-5, loss="rz")
    res = W.compare_starts(*test_run, xs, {"learned_extrap": net}, 12, warmup=3,
                           modes=("extrapolate", "learned_extrap"))
    ext, lrn = res["extrapolate"], res["learned_extrap"]
    assert lrn["relres_max"] <= 1e-8 and ext["relres_max"] <= 1e-8
    assert lrn["start_relres_geomean"] <= 0.5 * ext["start_relres_geomean"], res
    assert lrn["cycles_per_step"] <= ext["cycles_per_step"], res
    print(f"\nlearned correction vs extrapolated start: {res}")
    net.close()
