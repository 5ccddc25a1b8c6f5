"""The learned warm start inside the PIC step (pic_set_warm_unet).

 - A network with zero weights adds nothing to the initial guess: over several
   steps (recorded steps included) every integer moment, pid and iteration
   count equals the plain warm start's, and particles and potential agree
   within the store's parity bounds (two runs of either store differ in the
   last bits, since deposits sum in atomic order).
 - The warm start only moves the solve's starting point: with a random network
   and both solves run to a 1e-13 residual, the FP64 store still matches the CPU
   oracle (which starts from the previous potential) within the parity
   tolerances of tests/test_gpu_parity.py.
 - An instance configured with PIC_WARM_UNET and no network attached starts
   from the previous potential, as PIC_WARM_PREV.
 - What training gains: a network trained for a few hundred steps on samples
   of 32x32x64-cell runs leaves, on held-out samples, a smaller starting
   residual than the previous potential does, and in a held-out run the solve
   to the production residual (1e-8) still converges with it; the iterations of
   both forms are reported.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import unet_inputs as I
from paper_2606_05893_gb300 import workloads as W
from tests.gpu_compare import compare_integer_moments, compare_particles, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


def he_weights(pkg, seed):
    return np.concatenate([w.reshape(-1) for w in I.init_weights(pkg.UNET_WEIGHT_SHAPES, seed=seed)]).astype(np.float32)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_network_changes_nothing(pkg, precision):
    wl = W.config_tiny(seed=3)
    net = pkg.UNet(wl.nz, wl.ny, wl.nx, weights=np.zeros(pkg.unet_num_weights(), np.float32))
    a = pkg.Simulation(wl, precision=precision)
    b = pkg.Simulation(wl, precision=precision)
    pkg.pic_set_warm_unet(b.h, 0, net.net)
    for _ in range(6):
        a.step(1)
        b.step(1)
    ma, mb = a.moments(), b.moments()
    compare_integer_moments(mb, ma)
    assert ma["cg_iters"] == mb["cg_iters"]
    # deposits sum in atomic order (FP64 and FP32), which differs between any two
    # runs: the two agree within the store's parity bounds, integers exactly
    tol_x, tol_v, tol_phi = (1e-10 * max(wl.L), 1e-10, 1e-10) if precision == 0 else (1e-5 * wl.h, 1e-5, 1e-7)
    for sp in range(3):
        xa, va, pa = a.particles(sp)
        xb, vb, pb = b.particles(sp)
        oa, ob = np.argsort(pa), np.argsort(pb)
        assert np.array_equal(pa[oa], pb[ob])
        if pa.size:
            assert np.abs(xa[oa] - xb[ob]).max() <= tol_x
            assert np.abs(va[oa] - vb[ob]).max() <= tol_v * np.abs(va).max()
    assert rel_inf(b.phi(), a.phi()) <= tol_phi
    a.close()
    b.close()
    net.close()


def test_random_network_keeps_fp64_parity_with_oracle(pkg):
    wl = W.config_tiny(seed=5)
    net = pkg.UNet(wl.nz, wl.ny, wl.nx, weights=he_weights(pkg, 7))
    sim = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-13, cg_maxit=5000)
    pkg.pic_set_warm_unet(sim.h, 0, net.net)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    for _ in range(3):
        sim.step(1)
        ref.step(1)
    compare_integer_moments(sim.moments(), ref.moments())
    for sp in range(3):
        compare_particles(sim, ref, wl, sp, 1e-9, 1e-9)
    assert rel_inf(sim.phi(), ref.phi()) <= 1e-10
    assert sim.moments()["cg_resid_rel"] <= 1e-13
    sim.close()
    ref.close()
    net.close()


def test_trained_network_lowers_the_starting_residual(pkg):
    from paper_2606_05893_gb300 import warmstart as WS
    nx, ny, nz, h = 32, 32, 64, 2.5e-9
    runs = [W.config_warm_start(seed=s, n_preload=200_000, nx=nx, ny=ny, nz=nz, h=h, capacity_factor=2.0,
                                 r_emit=10e-9) for s in range(3)]
    held = W.config_warm_start(seed=50, n_preload=200_000, nx=nx, ny=ny, nz=nz, h=h, capacity_factor=2.0, r_emit=10e-9)
    net = pkg.UNet(nz, ny, nx, weights=he_weights(pkg, 0))
    train = WS.collect(runs, 30, 3, net)
    test = WS.collect([held], 10, 3, net)
    before = WS.residual_ratio(net, test, range(test.n))
    losses = WS.train(net, train, 400, lr=1e-3, seed=1)
    after = WS.residual_ratio(net, test, range(test.n))
    ev = WS.evaluate(held, net, 10, warmup=3)
    net.close()
    print(f"held-out starting residual / previous potential's: untrained {np.mean(before):.3f}, "
          f"trained {np.mean(after):.3f}; loss {np.mean(losses[:20]):.3e} -> {np.mean(losses[-20:]):.3e}; "
          f"iterations plain {np.mean(ev['plain']['iters']):.2f}, network {np.mean(ev['unet']['iters']):.2f}")
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    assert np.mean(after) < 0.8
    assert max(ev["unet"]["resid"]) <= 1e-8 and max(ev["plain"]["resid"]) <= 1e-8


def test_unet_mode_without_a_network_starts_from_the_previous_potential(pkg):
    # PIC_WARM_UNET marks the instance for a network; with none attached it is
    # PIC_WARM_PREV: the same integers and iterations, phi within FP64 parity
    wl = W.config_tiny(seed=4)
    a = pkg.Simulation(wl, precision=0, warm_start=pkg.PIC_WARM_PREV)
    b = pkg.Simulation(wl, precision=0, warm_start=pkg.PIC_WARM_UNET)
    for _ in range(4):
        a.step(1)
        b.step(1)
    ma, mb = a.moments(), b.moments()
    compare_integer_moments(mb, ma)
    assert ma["cg_iters"] == mb["cg_iters"]
    assert rel_inf(b.phi(), a.phi()) <= 1e-10
    a.close()
    b.close()
