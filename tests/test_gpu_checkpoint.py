"""Checkpoints: a run saved after n steps and resumed in a fresh handle
follows the run that was not interrupted.

The file holds the state, the forces of the last evaluation, the tangential
history, the evaluation index, the strain and the stress sums, so the resumed
run repeats the same arithmetic.  The force sums (atomics) may add in another
order, so the two runs agree to rounding grown over the remaining steps, not
bitwise.  A restore that dropped any of those parts would be off by far
more: the opening half kick of the resumed step moves U by dt F / m ~ 1e-4,
a lost tangential history changes contact forces at O(1).  Bars are 10-30
times the largest difference measured over two runs on a GB300 (FP64: x
8.9e-16, U 3.4e-14, W 8.6e-15, F 2.0e-14, history 1.4e-15; mixed: x
5.6e-10, U 1.1e-7, F 1.2e-7, history 5.6e-9)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# (x, U and W absolute; F normwise; history absolute) per precision
TOL = {"fp64": (1e-14, 1e-12, 2e-13, 5e-13, 3e-14),
       "mixed": (1e-8, 2e-6, 1e-6, 2e-6, 5e-8)}


def _args(w, precision):
    p = w.params
    return dict(precision=precision, eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
                shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
                torque_sign=p["torque_sign"], dt=p["dt"])


def _run(g, w, n):
    p = w.params
    g.step(n, p["shear_rate"], p["kT"], p["dt"], p["seed"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_follows_the_uninterrupted_run(tmp_path, precision, record):
    import paper_2307_13802_gb300 as susp

    w = workloads.make(600, 0.55, 100.0, 1.0, pack_seed=31, dyn_seed=32)
    path = str(tmp_path / "run.ckpt")
    a = susp.System(w.radii, w.box, **_args(w, precision))
    a.set_state(w.x, w.U, w.W)
    _run(a, w, 300)           # graph chunks and an eager tail
    k_saved = a.info()["k"]
    a.save(path)
    ij0, _ = a.history()
    assert len(ij0) > 20, "the run should hold tangential history"
    _run(a, w, 100)
    xa, Ua, Wa = a.state()
    Fa, Ta = a.forces()
    ija, xia = a.history()
    sa = a.stress()
    ia = a.info()

    b = susp.System(w.radii, w.box, **_args(w, precision))
    b.load(path)
    assert b.info()["k"] == k_saved
    _run(b, w, 100)
    xb, Ub, Wb = b.state()
    Fb, Tb = b.forces()
    ijb, xib = b.history()
    sb = b.stress()
    ib = b.info()

    tx, tu, tw, tf, th = TOL[precision]
    record("x", np.abs(xa - xb).max(), tx)
    record("U", np.abs(Ua - Ub).max(), tu)
    record("W", np.abs(Wa - Wb).max(), tw)
    record("F", np.abs(Fa - Fb).max() / np.abs(Fa).max(), tf)
    record("T", np.abs(Ta - Tb).max() / np.abs(Ta).max(), tf)
    record("hist", np.abs(xia - xib).max() if len(xia) else 0.0, th)
    assert ib["k"] == ia["k"] and ib["strain"] == pytest.approx(ia["strain"], abs=1e-15)
    assert np.abs(xa - xb).max() <= tx
    assert np.abs(Ua - Ub).max() <= tu
    assert np.abs(Wa - Wb).max() <= tw
    assert np.abs(Fa - Fb).max() <= tf * np.abs(Fa).max()
    assert np.abs(Ta - Tb).max() <= tf * np.abs(Ta).max()
    assert np.array_equal(ija, ijb)
    assert np.abs(xia - xib).max() <= th
    # stress sums continue across the checkpoint
    assert sb["samples"] == sa["samples"] > 300
    for key in ("contact", "lubrication", "brownian"):
        scale = np.abs(sa[key]).max()
        assert np.abs(sa[key] - sb[key]).max() <= 10 * tf * scale, key


def test_load_rejects_a_checkpoint_of_another_system(tmp_path):
    import paper_2307_13802_gb300 as susp

    w = workloads.make(300, 0.45, 10.0, 0.0, pack_seed=33, dyn_seed=34)
    path = str(tmp_path / "run.ckpt")
    a = susp.System(w.radii, w.box, **_args(w, "fp64"))
    a.set_state(w.x, w.U, w.W)
    _run(a, w, 10)
    a.save(path)
    radii = np.array(w.radii)
    radii[0] *= 1.01
    other = susp.System(radii, w.box, **_args(w, "fp64"))
    with pytest.raises(susp.SuspError, match="radii differ"):
        other.load(path)
    stiffer = susp.System(w.radii, w.box, **dict(_args(w, "fp64"), kn=2e4))
    with pytest.raises(susp.SuspError, match="model parameters differ"):
        stiffer.load(path)
    mixed = susp.System(w.radii, w.box, **_args(w, "mixed"))
    with pytest.raises(susp.SuspError, match="precision differs"):
        mixed.load(path)


def test_bad_checkpoint_files_are_reported(tmp_path):
    """Loading checks the file against the handle before it touches the
    device state."""
    import struct

    import paper_2307_13802_gb300 as s

    h = s.System([1.0] * 10, [30.0, 30.0, 30.0])
    with pytest.raises(s.SuspError, match="no state"):
        h.save(str(tmp_path / "x.ckpt"))
    with pytest.raises(s.SuspError, match="cannot open"):
        h.load(str(tmp_path / "missing.ckpt"))
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint at all" * 4)
    with pytest.raises(s.SuspError, match="not a checkpoint"):
        h.load(str(junk))
    # header: magic, N, R, precision, k, steps, dt, forces_valid, pad
    other = tmp_path / "other.ckpt"
    other.write_bytes(struct.pack("<8sqiiqqdii", b"SUSPCKP3", 11, 1, 0, 5, 5, 1e-4, 1, 0))
    with pytest.raises(s.SuspError, match="particle or replica count"):
        h.load(str(other))
    short = tmp_path / "short.ckpt"
    short.write_bytes(struct.pack("<8sqiiqqdii", b"SUSPCKP3", 10, 1, 0, 5, 5, 1e-4, 1, 0))
    with pytest.raises(s.SuspError, match="truncated"):
        h.load(str(short))
