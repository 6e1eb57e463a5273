import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def sc1_prepared():
    from paper_2109_08547_gb300 import synthetic
    import oracle
    wl = synthetic.workload_sc1()
    P = oracle.prepare(wl)
    return P


@pytest.fixture(scope="session")
def sc1_rates(sc1_prepared):
    import oracle
    return oracle.transition_rates(sc1_prepared)


@pytest.fixture(scope="session")
def sc1_full_prepared():
    """The one-band cubic model without point symmetry (brute-force full BZ)."""
    from paper_2109_08547_gb300 import synthetic
    import oracle
    return oracle.prepare(synthetic.workload_sc1(nsym_full=False))


@pytest.fixture(scope="session")
def sc1_full_rates(sc1_full_prepared):
    import oracle
    return oracle.transition_rates(sc1_full_prepared)
