"""The multi-core power iteration used for context timing agrees with the
oracle's PowItr (same iterations, same vector to rounding)."""
import numpy as np

import oracle as O
from oracle import context as C
import ppr_inputs as gen


def test_context_powitr_matches_oracle_powitr():
    rp, ci = gen.chung_lu(3000, 30000, 2.2, seed=5)
    og = O.Graph(rp, ci)
    cg = C.ContextGraph(rp, ci)
    assert C.threads() >= 1
    for s in gen.sources(og.n, 3, seed=9):
        pi_o, _, st = O.powitr(og, int(s), 0.2, 1e-8)
        pi_c, it = cg.powitr(int(s), 0.2, 1e-8)
        assert it == st["iterations"] == 83           # Eq. 6 at lambda = 1e-8, alpha = 0.2
        assert np.abs(pi_c - pi_o).sum() <= 1e-12
    cg.close()
