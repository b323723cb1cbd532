import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libadg.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def ff():
    from paper_2007_03678_gb300 import synth
    return synth.forcefield()


@pytest.fixture(scope="session")
def plain_inputs():
    """Plain workload: 40^3 maps from a 600-atom pseudo-receptor, 16+2 atom ligand, 3 torsions."""
    from paper_2007_03678_gb300 import synth
    return synth.workload_inputs(synth.PLAIN)


@pytest.fixture(scope="session")
def plain_maps(ff, plain_inputs):
    import oracle
    grid, rec, lig = plain_inputs
    return oracle.maps_build(ff, grid, rec)
