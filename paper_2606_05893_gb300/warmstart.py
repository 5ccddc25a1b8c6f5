"""Learned warm start of the Poisson solve: training samples from PIC runs,
training on the GPU with the library's own kernels, and the iterations the
trained network saves.

Every step of a sample, a training pass or an evaluation runs in the library
(include/unet.h, include/pic.h); this module only orders the calls and holds
device buffers (torch CUDA tensors).

Samples. A run steps its instance; after each step the potential of that step
and of the previous one give one pair: input (r / s, ramp) with r = A delta the
residual the previous potential leaves in this step's problem, target delta / s,
delta = phi_n - phi_{n-1} (unet_make_sample). That is what the warm start meets:
it starts the solve of step n from phi_{n-1} + s f(r / s, ramp).

Training. Adam, one sample per step, samples drawn in a seeded random order, on
the residual the warm start leaves, mean (r / s - A y)^2 over the unknown
planes (unet_train_step_residual): the solve's iteration count depends on that
residual. (The squared error against delta / s is the other choice; it weights
smooth components, which A shrinks, and leaves high-frequency errors, which A
amplifies up to twelvefold, so it does not lower the starting residual.)

Evaluation. Two instances of the same held-out workload, one with the plain warm
start (the previous step's potential) and one with the network, both solved to
the same relative residual; per step the iterations of the last solve
(pic_moments) and the CUDA-event times of the solve phase (pic_set_profiling).
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W


def _pkg():
    import paper_2606_05893_gb300 as pkg
    return pkg


class Samples:
    """N training pairs on the GPU: X (N, 2, D, H, W), T (N, D, H, W), scale s (N)."""

    def __init__(self, n, D, H, W):
        import torch
        self.X = torch.zeros((n, 2, D, H, W), dtype=torch.float32, device="cuda")
        self.T = torch.zeros((n, D, H, W), dtype=torch.float32, device="cuda")
        self.s = np.zeros(n)
        self.n = 0
        self.cap = n


def collect(wls, steps_per_run, skip, net, precision=None, samples=None, log=None):
    """Run every workload, skip `skip` steps, then take one sample per step."""
    import torch
    pkg = _pkg()
    precision = pkg.PIC_MIXED if precision is None else precision
    D, H, W = net.D, net.H, net.W
    if samples is None:
        samples = Samples(len(wls) * steps_per_run, D, H, W)
    nn = (D + 1) * H * W
    phi_a = torch.zeros(nn, dtype=torch.float64, device="cuda")
    phi_b = torch.zeros(nn, dtype=torch.float64, device="cuda")
    for wl in wls:
        assert (wl.nz, wl.ny, wl.nx) == (D, H, W)
        t0 = time.perf_counter()
        sim = pkg.Simulation(wl, precision=precision)
        sim.step(skip)
        pkg.pic_get_phi_device(sim.h, 0, phi_a.data_ptr())
        for _ in range(steps_per_run):
            if samples.n >= samples.cap:
                break
            sim.step(1)
            pkg.pic_get_phi_device(sim.h, 0, phi_b.data_ptr())
            i = samples.n
            samples.s[i] = net.make_sample(phi_b, phi_a, samples.X[i], samples.T[i])
            samples.n += 1
            phi_a, phi_b = phi_b, phi_a
        sim.close()
        if log:
            log(f"collected {samples.n} samples ({wl.name}, {time.perf_counter() - t0:.1f} s)")
    return samples


def train(net, samples, iters, lr=1e-3, lr_end=None, seed=0, log=None, every=100, objective="residual"):
    """Adam over the samples in a seeded random order; the learning rate decays
    geometrically from lr to lr_end (default lr / 10). objective "residual"
    minimises the scaled residual the warm start leaves (the quantity the solve
    then reduces), "target" the squared error against delta / s. Returns the
    losses."""
    rng = np.random.default_rng(seed)
    lr_end = lr / 10 if lr_end is None else lr_end
    losses = []
    order = rng.permutation(samples.n)
    k = 0
    t0 = time.perf_counter()
    for it in range(iters):
        if k == len(order):
            order, k = rng.permutation(samples.n), 0
        i = int(order[k])
        k += 1
        a = lr * (lr_end / lr) ** (it / max(iters - 1, 1))
        if objective == "residual":
            losses.append(net.train_step_residual(samples.X[i], a))
        else:
            losses.append(net.train_step(samples.X[i], samples.T[i], a))
        if log and (it + 1) % every == 0:
            log(f"iter {it + 1}: loss {np.mean(losses[-every:]):.4e} lr {a:.2e} ({time.perf_counter() - t0:.1f} s)")
    return losses


def residual_ratio(net, samples, idx):
    """||r - A s f(r/s)|| / ||r|| of the network's warm start on stored samples
    (host arithmetic on a few samples: a diagnostic, not the solve)."""
    out = []
    for i in idx:
        x0 = samples.X[i, 0].cpu().numpy().astype(np.float64)
        y = net.forward(samples.X[i]).cpu().numpy().astype(np.float64)
        y[-1] = 0.0
        Ay = 6 * y - np.roll(y, 1, 2) - np.roll(y, -1, 2) - np.roll(y, 1, 1) - np.roll(y, -1, 1)
        Ay[1:] -= y[:-1]
        Ay[:-1] -= y[1:]
        Ay[-1] = 0.0
        r = x0[:-1]
        out.append(float(np.linalg.norm(r - Ay[:-1]) / np.linalg.norm(r)))
    return out


def evaluate(wl, net, steps, warmup=5, precision=None, rtol=None):
    """Per-step iterations and solve-phase times of the plain warm start and of
    the network's, on two instances of the same workload."""
    import torch
    pkg = _pkg()
    precision = pkg.PIC_MIXED if precision is None else precision
    out = {}
    for mode in ("plain", "unet"):
        sim = pkg.Simulation(wl, precision=precision, cg_rtol=rtol)
        if mode == "unet":
            pkg.pic_set_warm_unet(sim.h, 0, net.net)
        sim.step(warmup)
        iters, resid = [], []
        pkg.pic_set_profiling(sim.h, True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            sim.step(1)
            m = sim.moments()
            iters.append(m["cg_iters"])
            resid.append(m["cg_resid_rel"])
        torch.cuda.synchronize()
        ph = pkg.pic_get_phase_times(sim.h, 0)
        pkg.pic_set_profiling(sim.h, False)
        out[mode] = {"iters": iters, "resid": resid, "solve_ms": ph["solve"][0] / steps,
                     "step_ms": sum(v[0] for v in ph.values()) / steps, "wall_s": time.perf_counter() - t0}
        sim.close()
    return out


def main(argv=None):
    import argparse
    import json

    import torch
    pkg = _pkg()
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start on the GPU")
    ap.add_argument("--runs", type=int, default=8)
    ap.add_argument("--steps", type=int, default=50, help="samples per run")
    ap.add_argument("--skip", type=int, default=5)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--n-preload", type=int, default=10_000_000)
    ap.add_argument("--eval-steps", type=int, default=40)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--out", default=None, help="write the trained weights here (.npy, FP32)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--forward-only", type=int, default=0, metavar="N",
                    help="only run N forward passes of a He-initialised network on a random 128x128x256 "
                         "input (for profilers) and exit")
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    prec = pkg.PIC_MIXED if a.precision == "mixed" else pkg.PIC_FP64
    log = lambda s: print(s, flush=True)  # noqa: E731
    from . import unet_inputs
    if a.forward_only:
        net = pkg.UNet(256, 128, 128)
        w = np.concatenate([w.reshape(-1) for w in unet_inputs.init_weights(pkg.UNET_WEIGHT_SHAPES, seed=a.seed)])
        net.set_weights(w.astype(np.float32))
        x = torch.from_numpy(unet_inputs.random_volume(2, 256, 128, 128, seed=a.seed).astype(np.float32)).cuda()
        for _ in range(a.forward_only):
            net.forward(x)
        torch.cuda.synchronize()
        net.close()
        log(f"{a.forward_only} forward passes")
        return 0
    wls = [W.config_warm_start(seed=a.seed + k, n_preload=a.n_preload) for k in range(a.runs)]
    wl0 = wls[0]
    net = pkg.UNet(wl0.nz, wl0.ny, wl0.nx)
    w0 = np.concatenate([w.reshape(-1) for w in unet_inputs.init_weights(pkg.UNET_WEIGHT_SHAPES, seed=a.seed)])
    net.set_weights(w0.astype(np.float32))
    samples = collect(wls, a.steps, a.skip, net, precision=prec, log=log)
    losses = train(net, samples, a.iters, lr=a.lr, seed=a.seed, log=log)
    ratio = residual_ratio(net, samples, range(0, samples.n, max(1, samples.n // 8)))
    log(f"warm-start residual / plain residual on training samples: {np.mean(ratio):.3f}")
    held = W.config_warm_start(seed=a.seed + 1000, n_preload=a.n_preload)
    ev = evaluate(held, net, a.eval_steps, precision=prec)
    res = {"train_losses_first_last": [float(np.mean(losses[:50])), float(np.mean(losses[-50:]))],
           "train_residual_ratio": float(np.mean(ratio)),
           "plain_iters_mean": float(np.mean(ev["plain"]["iters"])), "unet_iters_mean": float(np.mean(ev["unet"]["iters"])),
           "plain_solve_ms": ev["plain"]["solve_ms"], "unet_solve_ms": ev["unet"]["solve_ms"],
           "plain_step_ms": ev["plain"]["step_ms"], "unet_step_ms": ev["unet"]["step_ms"],
           "max_resid_unet": float(np.max(ev["unet"]["resid"]))}
    log(json.dumps(res))
    if a.out:
        np.save(a.out, net.weights())
    net.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
