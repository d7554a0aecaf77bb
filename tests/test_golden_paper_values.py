"""Host code against values the paper prints.

The fixtures in tests/golden/ copy printed numbers with their citations: the
tuned schedule constants (Sec. III.B, Eq. 5; Sec. III.D, Eq. 6), N_S and T_min
(Table I caption and columns), and the rows of Table I.  The paper prints no
worked example with intermediate values, so these are the only printed
numbers the implementation consumes; the tests check the schedule generators
and workload shapes against them and the closed forms they imply.
"""
import math
import pathlib

import numpy as np
import pytest

from paper_1710_09025_gb300 import schedules as S
from paper_1710_09025_gb300 import workloads as W

GOLDEN = pathlib.Path(__file__).parent / "golden"


def _value(text):
    if text.startswith("exp(") and text.endswith(")"):
        return math.exp(float(text[4:-1]))
    return float(text)


def _lines(name):
    for line in (GOLDEN / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            yield line.split()


def constants():
    out = {}
    for name, val, *cite in _lines("paper_constants.txt"):
        assert cite and cite[0] == "Sec.", name  # every value carries its citation
        out[name] = _value(val)
    return out


def table1():
    rows = []
    for t, D, L, R, T_min, NT, sched, M in _lines("table1_parameters.txt"):
        rows.append(dict(technique=t, D=int(D), L=int(L), R=int(R), T_min=float(T_min),
                         N_T=None if NT == "variable" else int(NT), schedule=sched, M=int(M)))
    return rows


def test_schedule_constants_are_the_printed_ones():
    c = constants()
    assert S.TSPL_ALPHA1 == c["tspl_alpha1"]
    assert S.TSPL_ALPHA2 == c["tspl_alpha2"]
    assert S.TSPL_BETA0 == c["tspl_beta0"]
    assert S.LBLT_TN_2D == c["lblt_TN_2D"]
    assert S.LBLT_TN_3D == c["lblt_TN_3D"]
    assert S.DPS_BETA0 == c["dps_beta0"]
    assert S.DPS_R == c["dps_r"]
    assert S.DPS_S == c["dps_S"]


def test_dps_with_the_printed_constants():
    # Eq. 6: R0 up to beta_0, then decreasing continuously to R0 / r at beta_max
    c = constants()
    beta_max, R0 = 1.0 / c["T_min"], 10 ** 6
    betas = S.lb(301, beta_max)
    R = S.dps_population(betas, R0, beta_max)
    assert np.all(R[betas <= c["dps_beta0"]] == R0)
    assert R[-1] == pytest.approx(R0 / c["dps_r"], rel=1e-12)
    assert np.all(np.diff(R[betas > c["dps_beta0"]]) < 0)
    assert S.dps_population([c["dps_beta0"] * (1 + 1e-12)], R0, beta_max)[0] == pytest.approx(R0, rel=1e-9)


def test_tspl_with_the_printed_constants():
    # Eq. 5: beta(0) = 0, beta(1) = beta_max, increasing, continuous at beta_0
    c = constants()
    beta_max = 1.0 / c["T_min"]
    b = S.tspl(301, beta_max)
    assert b[0] == 0.0 and b[-1] == pytest.approx(beta_max, rel=1e-12)
    assert np.all(np.diff(b) > 0)
    tau0 = (c["tspl_beta0"] / beta_max) ** (1.0 / c["tspl_alpha2"])
    a = c["tspl_beta0"] / tau0 ** c["tspl_alpha1"]
    assert a * tau0 ** c["tspl_alpha1"] == pytest.approx(beta_max * tau0 ** c["tspl_alpha2"], rel=1e-12)


def test_lblt_with_the_printed_tuning_temperatures():
    c = constants()
    for TN in (c["lblt_TN_2D"], c["lblt_TN_3D"]):
        b = S.lblt(101, c["T_min"], TN)
        assert len(b) == 101 and b[0] == 0.0
        assert b[50] == pytest.approx(1.0 / TN, rel=1e-15)           # end of the linear-in-beta half
        assert 1.0 / b[-1] == pytest.approx(c["T_min"], rel=1e-15)   # linear in T down to T_min
        assert np.allclose(np.diff(1.0 / b[51:]), np.diff(1.0 / b[51:])[0], rtol=1e-9)


def test_table1_shapes_and_the_workloads():
    c = constants()
    rows = table1()
    assert len(rows) == 25
    assert {r["technique"] for r in rows} == {"SSM", "AS", "NT", "DPS", "CA"}
    for r in rows:
        assert r["T_min"] == c["T_min"]
        if r["N_T"] is not None:
            b = S.lb(r["N_T"], 1.0 / r["T_min"])
            assert len(b) == r["N_T"] and b[0] == 0.0 and b[-1] == 1.0 / c["T_min"]
    # every workload here uses the printed N_S; the 3D +-J ones anneal to T_min,
    # and where Table I has a linear-in-beta row of the same L, with its N_T
    lb_rows = {(r["D"], r["L"]): r["N_T"] for r in rows if r["schedule"] == "LB" and r["N_T"]}
    for name, w in W.WORKLOADS.items():
        assert w["n_sweeps"] == c["n_sweeps"], name
        if w["D"] == 3 and w["kind"] == 0:
            assert w["beta_max"] == 1.0 / c["T_min"], name
            if (3, w["L"]) in lb_rows:
                assert w["n_temps"] == lb_rows[(3, w["L"])], name
