"""The CSR graph check (a guard of this library, not part of the paper): a
valid graph passes, each kind of corruption is reported by name, and with
ENS_CHECK=1 a solve on a corrupted graph returns ENS_EINVAL before any kernel
reads through it.  The corruptions only ever reach the check kernel, which
reads rowptr[0..J] and colidx[0..nnz) whatever they hold."""
import os

import numpy as np
import pytest
import torch

from gpu_util import Case
from paper_1705_02003_gb300 import ens, inputs

pytestmark = pytest.mark.gpu


def _graph(h, kind="q1", n=12):
    prob = ens.problem(kind, n, {"fd5": 2, "q1": 4, "fd7": 6}[kind], 4.0)
    J, nnz = ens.ens_problem_size(prob)
    rp = torch.empty(J + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(nnz, dtype=torch.int32, device="cuda")
    ens.ens_pattern(h, prob, rp, ci)
    return J, nnz, rp, ci


def test_valid_graphs_pass(ens_lib):
    h = ens.Handle(0)
    for kind in ("fd5", "q1", "fd7"):
        J, nnz, rp, ci = _graph(h, kind, 10)
        ens.ens_check_pattern(h, J, nnz, rp, ci)
    h.close()


@pytest.mark.parametrize("what,match", [("colidx_high", "column index"), ("colidx_neg", "column index"),
                                        ("rowptr_order", "decreases"), ("rowptr_end", "rowptr\\[J\\]"),
                                        ("rowptr_range", "outside \\[0, nnz\\]")])
def test_each_corruption_is_reported(ens_lib, what, match):
    h = ens.Handle(0)
    J, nnz, rp, ci = _graph(h)
    if what == "colidx_high":
        ci[17] = J
    elif what == "colidx_neg":
        ci[nnz - 1] = -1
    elif what == "rowptr_order":
        rp[40] = rp[42]  # rowptr[40] > rowptr[41]
    elif what == "rowptr_end":
        rp[J] = nnz - 1
    else:
        rp[J // 2] = nnz + 5
    with pytest.raises(ens.EnsError, match=match):
        ens.ens_check_pattern(h, J, nnz, rp, ci)
    h.close()


def test_checked_solve_refuses_a_bad_graph(ens_lib):
    saved = os.environ.get("ENS_CHECK")
    os.environ["ENS_CHECK"] = "1"
    try:
        h = ens.Handle(0)
    finally:
        if saved is None:
            os.environ.pop("ENS_CHECK", None)
        else:
            os.environ["ENS_CHECK"] = saved
    xi = inputs.draws(8, 4, seed=3)
    c = Case(h, "q1", 12, 4, 4.0, 8, xi)
    good = c.solve(1e-8, 5000)  # a valid graph solves as usual under the check
    assert np.all(good["status"] == ens.LANE_CONVERGED)
    c.colidx[5] = c.J  # one past the last column: refused before any kernel reads p through it
    with pytest.raises(ens.EnsError, match="column index"):
        c.solve(1e-8, 5000)
    h.close()
