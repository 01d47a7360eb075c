"""The dissolution case of Sec. 4.3 on the oracle: a bubble in a liquid
without dissolved gas loses gas through Henry's law at its interface."""
import numpy as np

from paper_1908_04262_gb300 import workloads as W


def test_bubble_dissolves_into_gas_free_liquid(oracle_mod):
    cfg, c, r = W.dissolution_2d()
    s = oracle_mod.OracleSim(cfg)
    s.nucleate(c, r)

    def state():
        b = s.bubbles()
        i = int(np.flatnonzero(b["atm"] == 0)[0])
        L = s.ledger()
        return b["volume"][i], b["mass"][i], L[3], L[3] + L[4] + L[5] - L[6]

    V, m, dissolved, total = [], [], [], []
    for k in range(7):
        if k:
            s.step(500)
        v, mm, d, t = state()
        V.append(v)
        m.append(mm)
        dissolved.append(d)
        total.append(t)
    V, m, dissolved, total = map(np.asarray, (V, m, dissolved, total))
    # the bubble shrinks and loses gas at every sample, the liquid gains gas
    assert np.all(np.diff(V) < 0) and np.all(np.diff(m) < 0)
    assert np.all(np.diff(dissolved) > 0)
    assert V[-1] < 0.9 * V[0]
    # gas is accounted for: dissolved + bubbles + exchanged with the outside
    # (the headspace also dissolves into the liquid) - source is conserved to
    # round-off (the flux of Eq. gascurrent is the exchange at the gas links,
    # and cells changing between gas and interface carry their dissolved gas)
    assert np.max(np.abs(total - total[0])) < 1e-11 * (dissolved[-1] - dissolved[0])
