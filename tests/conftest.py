import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def eq_mothers_256():
    """Equilibrium mother states of the N=256 bulk system (Example 1 state
    point), computed by the oracle: 8 independent mothers, each thermalised
    4000 steps, then 6 states 200 steps apart.  Returns (Bulk, states
    [48, 6, N], alphas [48])."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2312_02990_gb300 import inputs

    N = 256
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))

    def one(k):
        s0 = inputs.initial_state(N, inputs.BASE_SEED + k)
        return oracle.mother(b, s0, n_eq=4000, n_states=6, spacing=200)

    with ThreadPoolExecutor(8) as ex:
        res = list(ex.map(one, range(8)))
    states = np.concatenate([r[0] for r in res])
    alphas = np.concatenate([r[1] for r in res])
    return b, states, alphas
