"""A nested-dissection order against the library's minimum-degree order, on the
host-only plan: the dissection order is a valid permutation that the analysis
accepts, and on these KKT graphs it makes the assembly tree taller and the
factors larger (its separators are chained into levels of at most 16 pivots),
which is why the library keeps minimum degree. Printed with -s."""
import numpy as np
import pytest

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, WORKLOADS, make_grid
from nd_order import nested_dissection


@pytest.mark.parametrize("name", ["grid200", pytest.param("northeast25k", marks=pytest.mark.slow)])
def test_dissection_order_against_minimum_degree(name):
    w = WORKLOADS[name]
    pat = KKTPattern(make_grid(1, w["n_bus"], w["n_branch"], w["n_gen"]))
    q = nested_dissection(pat)
    assert np.array_equal(np.sort(q), np.arange(pat.n))
    md = K.plan(pat.rowptr, pat.colidx)
    nd = K.plan(pat.rowptr, pat.colidx, user_perm=q)
    for label, p in (("minimum degree", md), ("nested dissection", nd)):
        print("%s %-17s levels %3d  fronts %6d  max front %4d  nnz(L+U) %9d  flops %.1f M"
              % (name, label, p["n_levels"], p["n_fronts"], p["max_front"], p["nnz_lu"], p["flops"] / 1e6))
    assert nd["nnz_lu"] >= md["nnz_lu"] and nd["flops"] >= md["flops"]
