"""Shared test configuration.

Markers: ``gpu`` tests need a CUDA device and the built library; everything
else runs on the CPU in a few minutes.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libsf.so")


@pytest.fixture(scope="session")
def oracle():
    """The FP64 oracle package.

    SF_ORACLE_DIR points the fixture at another copy of the package; the
    mutation test uses it to run the pins against oracles with planted slips.
    """
    alt = os.environ.get("SF_ORACLE_DIR")
    if alt:
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "oracle_under_test", os.path.join(alt, "__init__.py"),
            submodule_search_locations=[alt])
        orc = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(orc)
    else:
        import oracle as orc
    orc.build()
    return orc
