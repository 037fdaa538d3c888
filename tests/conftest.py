import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


def _two_sphere_capacitance(a: float, d: float, terms: int = 200) -> float:
    """Capacitance (in units where an isolated sphere of radius a has a) of two
    spheres of radius a, centres d apart, held at the same potential: the
    method of images.  A charge q at offset x from one centre (towards the
    other) has its image -q a / (d - x) in the other sphere, at offset
    a^2 / (d - x) from that sphere's centre; by symmetry both spheres carry
    the same charges, starting from a at each centre."""
    q, x, tot = a, 0.0, 0.0
    for _ in range(terms):
        tot += q
        q, x = -q * a / (d - x), a * a / (d - x)
    return 2.0 * tot


@pytest.fixture(scope="session")
def two_sphere_capacitance():
    return _two_sphere_capacitance
