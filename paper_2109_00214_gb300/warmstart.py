"""Host-side orchestration of the learned Poisson warm start: collecting
training pairs from simulations, the training loop and the comparison of the
solve's starting points.  Every computation runs in the library's kernels
(pd_warmstart_pairs, pd_net_loss_grad, pd_net_adam, pd_step); this module
only moves batches between device tensors and calls them.
"""
import numpy as np

from . import Ensemble, Net, Simulation


def collect_pairs(cfgs, loads, xs, n_pairs, every=2, warmup=2, kinds=("absolute",), device="cuda"):
    """Advance the runs `cfgs` (all one grid shape) as one ensemble and take
    (x, t) pairs of each of `kinds` every `every` steps: returns {kind: (x, t)}
    with device tensors of shape [runs, n_pairs, H, W] (float32)."""
    import torch
    H, W = cfgs[0]["nz"] + 1, cfgs[0]["nr"] + 1
    for c in cfgs:
        assert (c["nz"] + 1, c["nr"] + 1) == (H, W)
    ens = Ensemble(cfgs, xs, device=device)
    for r, parts in enumerate(loads):
        ens.load_run(r, parts)
    R = len(cfgs)
    out = {k: (torch.empty((R, n_pairs, H, W), dtype=torch.float32, device=device),
               torch.empty((R, n_pairs, H, W), dtype=torch.float32, device=device)) for k in kinds}
    ens.step(warmup)
    for j in range(n_pairs):
        ens.step(every)
        for k in kinds:
            x, t = ens.warmstart_pairs(k)
            out[k][0][:, j] = x.view(R, H, W)
            out[k][1][:, j] = t.view(R, H, W)
    ens.synchronize()
    ens.close()
    return out


def train(net, sets, iters, batch, lr=1e-3, lr_final=1e-4, seed=0, log_every=0, loss="mse"):
    """Adam on mini-batches drawn from `sets` (a list of (X, T) tensors of
    shape [n, H, W], one per grid shape, used in turn).  The learning rate
    decays geometrically from lr to lr_final.  `loss`: "mse" against the
    targets T, or "rz", the residual of Eq. (8) that the start leaves
    (pd_net_loss_grad_rz; T unused).  Returns the loss history
    [(iteration, loss)] taken every `log_every` iterations."""
    import torch
    from . import pd_net_loss_grad, pd_net_loss_grad_rz
    g = torch.Generator(device=sets[0][0].device)
    g.manual_seed(seed)
    hist = []
    for it in range(iters):
        X, T = sets[it % len(sets)]
        b = batch[it % len(sets)] if isinstance(batch, (list, tuple)) else batch
        idx = torch.randint(0, X.shape[0], (b,), device=X.device, generator=g)
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
        # the loss is read back (a synchronisation) only on logged iterations
        if loss == "rz":
            lv, _ = pd_net_loss_grad_rz(net.h, xb.data_ptr(), b, X.shape[1], X.shape[2], want, False)
        else:
            lv, _ = pd_net_loss_grad(net.h, xb.data_ptr(), tb.data_ptr(), b, X.shape[1], X.shape[2], want, False)
        net.adam(lr=lr * (lr_final / lr) ** (it / max(iters - 1, 1)))
        if want:
            hist.append((it, lv))
    return hist


def test_loss(net, X, T, batch=4, loss="mse"):
    """Mean loss over the pairs of (X, T) ([n, H, W] device tensors)."""
    tot, n = 0.0, 0
    for s in range(0, X.shape[0], batch):
        xb, tb = X[s:s + batch].contiguous(), T[s:s + batch].contiguous()
        lv, _ = net.loss_grad_rz(xb) if loss == "rz" else net.loss_grad(xb, tb)
        tot += lv * xb.shape[0]
        n += xb.shape[0]
    return tot / n


def compare_starts(cfg, parts, xs, nets, steps, warmup=2, modes=("previous", "cold", "learned"), device="cuda"):
    """Step the run `cfg` from the same start under each warm-start mode
    (host-checked multigrid to the configured tolerance) and report, per
    mode, the multigrid cycles per step, the step time (CUDA events) and the
    geometric mean of the solves' starting residuals.
    `nets` maps the learned modes to their networks."""
    import torch
    out = {}
    for mode in modes:
        sim = Simulation(cfg, xs, device=device)
        sim.load(parts)
        sim.step(warmup)
        sim.set_warm_start(mode, nets.get(mode))
        sim.synchronize()
        cyc, ms, r0, worst = [], [], [], 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(steps):
            e0.record(sim.stream)
            sim.step(1)
            e1.record(sim.stream)
            sc = sim.scalars()
            cyc.append(sc["poisson_cycles"])
            r0.append(sc["poisson_relres0"])
            worst = max(worst, sc["poisson_relres_max"])
            ms.append(e0.elapsed_time(e1))
        out[mode] = {"cycles_per_step": float(np.mean(cyc)), "ms_per_step": float(np.mean(ms)),
                     "relres_max": worst, "start_relres_geomean": float(np.exp(np.mean(np.log(np.maximum(r0, 1e-300)))))}
        sim.close()
    return out
