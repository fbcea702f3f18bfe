"""Host logic of the reuse of f across time steps (paper Sec. 4.2): the
library's decision (vet.reuse_decision) against the oracle's decision on
seeded triples, ages and tolerances, including non-finite changes and
triples on the tolerance boundary."""
import numpy as np

from oracle import field_change as fc
from paper_2202_08778_gb300 import vet


def test_decision_matches_the_oracle():
    rng = np.random.default_rng(9)
    for _ in range(20000):
        triple = np.float32(rng.lognormal(-4.0, 2.0, 3))
        r = rng.random()
        if r < 0.05:
            triple[rng.integers(2)] = np.inf
        elif r < 0.1:
            triple[rng.integers(2)] = np.nan
        tol_tau, tol_S = (float(np.float32(x)) for x in rng.lognormal(-4.0, 1.5, 2))
        if rng.random() < 0.1:                    # exactly on the boundary
            triple[0] = np.float32(tol_tau)
        age, first, max_age = int(rng.integers(0, 10)), bool(rng.random() < 0.1), int(rng.integers(1, 10))
        want = fc.recompute(triple, age, first, tol_tau, tol_S, max_age)
        assert vet.reuse_decision(triple, age, first, tol_tau, tol_S, max_age) == want
