"""susp_pair_stress_noalloc: the pair stresses for callers that cannot
allocate device memory, checked against the handle-based evaluation.

The caller owns every buffer (here: torch tensors on cuda:0) and the call
keeps its scratch in a fixed device array, so it must give the handle's
answer on every call, including a second call in a row that finds the
previous call's partial sums still in that array."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-11  # same double-precision arithmetic, different summation order


def _relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


def test_noalloc_pair_stress_matches_the_handle():
    import torch

    import paper_2307_13802_gb300 as susp

    w = workloads.make(3000, 0.56, 10.0, 0.0, pack_seed=91, dyn_seed=92)
    w.x = w.x * 0.985          # compress a little: many overlapping pairs
    w.L = w.L * 0.985
    p = w.params
    kw = dict(precision="fp64", eta=p["eta"], kn=p["kn"], shear_rate=p["shear_rate"],
              kT=p["kT"], seed=p["seed"], dt=p["dt"], xi_min=p["xi_min"],
              xi_max=p["xi_max"], torque_sign=p["torque_sign"])
    k, strain = 11, 0.3
    g = susp.System(w.radii, w.box, **kw)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(k, strain)
    g.evaluate()
    ref = g.stress()
    ij = g.pairs()
    x, U, W = g.state()        # the wrapped state the handle evaluated
    assert len(ij) > 1000

    dev = torch.device("cuda:0")
    tx = torch.tensor(x, dtype=torch.float64, device=dev).contiguous()
    tU = torch.tensor(U, dtype=torch.float64, device=dev).contiguous()
    tW = torch.tensor(W, dtype=torch.float64, device=dev).contiguous()
    tr = torch.tensor(w.radii, dtype=torch.float64, device=dev).contiguous()
    tij = torch.tensor(ij, dtype=torch.int32, device=dev).contiguous()
    out = torch.empty(27, dtype=torch.float64, device=dev)
    params = susp.default_params(**kw)
    box = np.ascontiguousarray(w.box, dtype=np.float64)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call(npairs):
        return susp.lib.susp_pair_stress_noalloc(
            w.N, tx.data_ptr(), tU.data_ptr(), tW.data_ptr(), tr.data_ptr(), npairs,
            tij.data_ptr(), box.ctypes.data_as(C.POINTER(C.c_double)), strain,
            C.byref(params), p["dt"], k, out.data_ptr(), stream)

    for _ in range(2):
        out.fill_(float("nan"))
        assert call(len(ij)) == susp.SUSP_OK, susp.lib.susp_create_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(3, 3, 3)
        for c, key in enumerate(("contact", "lubrication", "brownian")):
            assert np.all(np.isfinite(got[c]))
            assert _relerr(got[c], ref[key]) <= RTOL, key

    # sizes beyond the static scratch are refused before any work is issued
    assert call((1 << 21) + 1) == susp.SUSP_EINVAL
    assert "SUSP_NOALLOC_MAX_PAIRS" in susp.lib.susp_create_error().decode()
