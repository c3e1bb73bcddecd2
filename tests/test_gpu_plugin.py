"""PyTorch as the source of device memory and input tensors.

A handle whose device memory comes from PyTorch's caching allocator (through
susp_set_allocator) and whose state is loaded from CUDA tensors (through
susp_set_state_device) computes what a handle on the library's own
cudaMalloc memory, loaded from host arrays, computes: the same kernels on
the same numbers, so forces, torques and stresses agree to the summation
order of the atomics (measured ~1e-15; bar 1e-11)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _kw(w, precision):
    p = w.params
    return dict(precision=precision, eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
                shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
                torque_sign=p["torque_sign"], dt=p["dt"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_torch_memory_and_tensors_give_the_same_run(precision, record):
    import torch

    import paper_2307_13802_gb300 as susp

    w = workloads.make(2000, 0.55, 10.0, 1.0, pack_seed=201, dyn_seed=202)
    p = w.params
    dev = torch.device("cuda", 0)
    xt = torch.tensor(w.x, dtype=torch.float64, device=dev)
    Ut = torch.tensor(w.U, dtype=torch.float64, device=dev)
    Wt = torch.tensor(w.W, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(dev)

    a = susp.System(w.radii, w.box, **_kw(w, precision))
    alloc, release = susp.torch_allocator(dev)
    a.set_allocator(alloc, release)
    a.set_state_device(xt.data_ptr(), Ut.data_ptr(), Wt.data_ptr())
    held = a.info()["device_bytes"]
    torch.cuda.synchronize()
    # the handle's memory is PyTorch's: the caching allocator accounts for it
    assert torch.cuda.memory_allocated(dev) - base >= held > 0

    b = susp.System(w.radii, w.box, **_kw(w, precision))
    b.set_state(w.x, w.U, w.W)
    for s in (a, b):
        s.step(150, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    Fa, Ta = a.forces()
    Fb, Tb = b.forces()
    sa, sb = a.stress(), b.stress()
    eF = np.abs(Fa - Fb).max() / np.abs(Fb).max()
    eT = np.abs(Ta - Tb).max() / np.abs(Tb).max()
    es = max(np.abs(sa[k] - sb[k]).max() / np.abs(sb[k]).max()
             for k in ("contact", "lubrication", "brownian"))
    tol = 1e-11 if precision == "fp64" else 1e-5
    record("force", eF, tol)
    record("torque", eT, tol)
    record("stress", es, tol)
    assert eF <= tol and eT <= tol and es <= tol
    a.close()
    torch.cuda.synchronize()
    # destroying the handle hands every block back
    assert torch.cuda.memory_allocated(dev) == base
