"""The swarm hyper-parameters of Table III as the library's swarm uses them:
the paper's columns (eps of M_c, eta, beta, lambda, iota, psi, f_low, e0)
mapped onto this build's parameter order (M_c, q, f0, lambda, beta, iota,
psi, e0) -- eta's minimum speed applied to q and f_low's to f0 -- and the rung
chosen for a segment count."""
import json
import os

import pytest

from paper_2408_13170_gb300 import scstat

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_pso_hyper.json")


def test_rows_are_the_papers_in_parameter_order():
    g = json.load(open(GOLDEN))
    col = {c: i for i, c in enumerate(g["columns"])}
    order = ["eps_Mc", "eps_eta", "eps_flow", "eps_lambda", "eps_beta", "eps_iota", "eps_psi",
             "eps_e0"]
    assert sorted(int(n) for n in g["rows"]) == sorted(scstat.TABLE3_HYPER)
    for n, row in g["rows"].items():
        om, pp, pg, eps = scstat.TABLE3_HYPER[int(n)]
        assert (om, pp, pg) == (row[col["Omega"]], row[col["Phi_P"]], row[col["Phi_G"]])
        assert tuple(eps) == tuple(row[col[c]] for c in order)


@pytest.mark.parametrize("N,rung", [(100, 100), (2048, 100), (75, 100), (60, 50), (30, 50),
                                    (20, 10), (10, 10), (5, 1), (1, 1)])
def test_closest_rung_ties_to_the_larger(N, rung):
    assert scstat.table3_hyper(N) == scstat.TABLE3_HYPER[rung]
