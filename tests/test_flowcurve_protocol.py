"""The flow-curve harness lays out Table 1's protocol (Sec. IV.D): checked on
the CPU against the table's printed shear rates and thermal energies."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_protocol_reproduces_the_printed_rates_and_temperatures():
    from paper_2307_13802_gb300 import flowcurve

    rows = np.loadtxt(os.path.join(GOLDEN, "table1_parameters.txt"))
    # Table 1 runs at rate0 = 0.009 with eta = 0.1, a = 1
    for pe, rate, kT, a, rho, kn, eta in rows:
        r, t = flowcurve.table1_point(pe, rate0=0.009, eta=eta, a=a)
        # printed to two significant figures
        assert r == pytest.approx(rate, rel=0.06), (pe, r, rate)
        assert t == pytest.approx(kT, rel=0.06), (pe, t, kT)
    # the switch: rate varies below Pe = 1, kT above
    r1, t1 = flowcurve.table1_point(0.5)
    r2, t2 = flowcurve.table1_point(5.0)
    assert r1 == 0.5 and t2 == pytest.approx(t1 / 5.0) and r2 == 1.0


def test_equal_volume_mixing():
    from paper_2307_13802_gb300 import flowcurve

    for N in (500, 1000, 12345):
        ns, nl = flowcurve.equal_volume_counts(N)
        assert ns + nl == N
        # volumes ns * 1 and nl * 1.4^3 as equal as integer counts allow
        assert abs(ns - nl * 1.4 ** 3) <= 1.4 ** 3
