"""Per-term residual parity against the oracle (FP64 and FP32).  The terms
of the residual are switched on one after another through the flow
parameters, which switch them off identically in both codes: inviscid
fluxes only (Re = inf, C_s = 0, k2 = k4 = 0), + Turkel-Vatsa dissipation
(k2, k4), + molecular viscous and heat fluxes (finite Re), + Smagorinsky /
Eidson SGS terms (C_s).  A mistake confined to one term shows as the first
stage whose residual departs from the oracle's."""
import math

import numpy as np
import pytest

import oracle
from helpers import to_oracle
from paper_2212_12365_gb300 import inputs as I
from paper_2212_12365_gb300 import les

pytestmark = pytest.mark.gpu

TERMS = [
    ("inviscid", dict(Re=math.inf, Cs=0.0, k2=0.0, k4=0.0)),
    ("+dissipation", dict(Re=math.inf, Cs=0.0, k2=0.25, k4=0.016)),
    ("+viscous", dict(Re=400.0, Cs=0.0, k2=0.25, k4=0.016)),
    ("+sgs", dict(Re=400.0, Cs=0.17, k2=0.25, k4=0.016)),
]

GRIDS = {
    "wavy_box": lambda: I.wavy_box_grid((14, 11, 9), amp=0.06, bc=(1, 3, 1, 1, 1, 1)),
    "jet_ragged": lambda: I.jet_grid(37, 23, 19, 8.0, 6.0, 6.0, 0.15, 0.18),
    "wavy_periodic": lambda: I.wavy_periodic_grid((13, 11, 9), amp=0.2),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_12365_gb300 import build
    build.build()


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("prec,tol", [(les.LES_FP64, 1e-13), (les.LES_FP32, 1e-5)])
def test_residual_term_by_term(grid, prec, tol):
    spec = GRIDS[grid]()
    prim = I.smooth_random_primitives(spec, 23, amp=0.08)
    report = []
    for name, kw in TERMS:
        fp = I.FlowParams(**kw)
        g, p = to_oracle(spec, fp)
        m = oracle.metrics(g)
        q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, prim, True), 0)
        r_or = oracle.rhs(g, p, m, q)
        s = les.Solver(spec, fp, prec)
        s.set_state(prim)
        r = s.rhs()
        s.close()
        # per field, relative to the field's residual scale (a field whose
        # residual vanishes for this term set is held to the largest scale)
        scale = np.maximum(np.abs(r_or).max(axis=1), 1e-3 * np.abs(r_or).max())[:, None]
        err = (np.abs(r - r_or) / scale).max(axis=1)
        report.append((name, err.max()))
        assert np.all(err <= tol), (grid, name, err)
    print(grid, "precision", prec, "max error per term set:", report)
