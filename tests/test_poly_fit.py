"""The HH_PREC_POLY rate tables (hh_poly_fit, a host computation of the
library: no GPU) against the FP64 oracle's own rate code: at random V over
the whole tabulated range, every gate's p_inf and 1 - e^{-dt/tau} evaluated
from the table agree with oracle.gate_inf_tau to the stated bound, and the
table covers [HH_POLY_V_LO, HH_POLY_V_HI) with the interval it reports."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp


def _gates(model):
    return [g for ch in model["channels"] for g in ch["gates"]]


@pytest.mark.parametrize("name", ["hh1952", "multi6"])
@pytest.mark.parametrize("dt", [0.01, 0.025])
def test_table_matches_oracle_rates(name, dt):
    model = inp.MODELS[name]
    h, v_lo, err, c = hh.hh_poly_fit(model, dt)
    n = c.shape[0]
    assert v_lo == hh.HH_POLY_V_LO and abs(v_lo + n * h - hh.HH_POLY_V_HI) < 1e-4
    assert err <= hh.HH_POLY_REL_ERR
    rng = np.random.default_rng(3)
    V = np.concatenate([rng.uniform(hh.HH_POLY_V_LO, hh.HH_POLY_V_HI, 400),
                        [-40.0, -55.0, -8.9, -35.0, -65.0]])  # removable points and rest
    Ca = 0.3
    worst = 0.0
    for v in V:
        u = (v - v_lo) / h
        j = min(int(math.floor(u)), n - 1)
        x = u - j
        for q, g in enumerate(_gates(model)):
            inf_r, tau_r = oracle.gate_inf_tau(g, v, Ca)
            E_r = -math.expm1(-dt / tau_r)
            for f, ref in ((0, inf_r), (1, E_r)):
                if f == 0 and g["kind"] == "ca":
                    assert not c[j, q, 0].any()
                    continue
                a = c[j, q, f].astype(np.float64)
                got = a[0] + x * (a[1] + x * (a[2] + x * a[3]))
                e = abs(got - ref) / max(abs(ref), 1e-7)
                worst = max(worst, e)
                assert e <= 1e-6, (name, v, q, f, got, ref)
    print(f"{name} dt {dt}: interval {h} mV, fit error {err:.2e}, against the oracle {worst:.2e}")


def test_fit_rejects_invalid_model():
    m = dict(inp.CLASSIC_HH, C_m=-1.0)
    with pytest.raises(hh.HHError) as e:
        hh.hh_poly_fit(m, 0.01)
    assert e.value.status == hh.HH_EINVAL
