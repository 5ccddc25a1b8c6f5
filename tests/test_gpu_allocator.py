"""Device memory from the caller's allocator (pic_set_allocator) on the GPU.

With PyTorch's caching allocator behind the library, an FP64 run matches the
oracle as with cudaMalloc (integer moments exact, particles, rho and phi within
1e-9 after several steps); every buffer the handle took is handed back when it
is destroyed (as many frees as allocations, torch's allocated bytes back where
they were); the allocator cannot change while a handle is alive; a U-Net handle
takes and returns its memory the same way.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_05893_gb300 import workloads as W
from tests.test_gpu_parity import full_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2606_05893_gb300 as p
    p.load_library()
    return p


@pytest.fixture
def counted(pkg):
    import torch
    log = {"alloc": 0, "free": 0, "live": set()}

    def alloc(nbytes):
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        log["alloc"] += 1
        log["live"].add(ptr)
        return ptr

    def free(ptr):
        log["free"] += 1
        log["live"].discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    pkg.pic_set_allocator(alloc, free)
    try:
        yield log
    finally:
        pkg.pic_set_allocator()


def test_run_on_torch_memory_matches_oracle(pkg, counted):
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    wl = W.config_tiny(seed=5)
    sim = pkg.Simulation(wl, precision=pkg.PIC_FP64, cg_rtol=1e-13, cg_maxit=5000)
    ref = O.Oracle(wl, cg_rtol=1e-13)
    assert counted["alloc"] > 20 and torch.cuda.memory_allocated() > base
    with pytest.raises(pkg.PicError):  # memory must go back to the allocator it came from
        pkg.pic_set_allocator()
    for _ in range(6):
        sim.step()
        ref.step()
    mg, _ = full_compare(sim, ref, wl, tol=1e-9)
    assert sum(mg["injected"]) > 0
    sim.close()
    ref.close()
    torch.cuda.synchronize()
    assert counted["free"] == counted["alloc"] and not counted["live"]
    assert torch.cuda.memory_allocated() == base


def test_unet_handle_on_torch_memory(pkg, counted):
    net = pkg.unet_create(16, 16, 16)
    n = counted["alloc"]
    assert n > 0
    pkg.unet_destroy(net)
    assert counted["free"] == n and not counted["live"]
