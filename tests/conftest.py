import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

_JOBS = None


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")
    config.addinivalue_line("markers", "oracle_jobs(*names): uses full-size oracle solves run in worker processes")


@pytest.hookimpl(trylast=True)
def pytest_collection_modifyitems(session, config, items):
    """Start the full-size oracle solves the selected tests need (after deselection, before
    any test runs, so before the first GPU call): they run in spawned worker processes
    while the other tests use the GPU."""
    global _JOBS
    if config.option.collectonly:
        return
    names = []
    for it in items:
        for mk in it.iter_markers("oracle_jobs"):
            names.extend(n for n in mk.args if n not in names)
    if names:
        import oracle_jobs

        _JOBS = oracle_jobs.Jobs(names)


def pytest_unconfigure(config):
    global _JOBS
    if _JOBS is not None:
        _JOBS.close()
        _JOBS = None


@pytest.fixture(scope="session")
def jobs():
    assert _JOBS is not None, "no oracle jobs were started"
    return _JOBS


@pytest.fixture(scope="session")
def orc():
    import oracle

    o = oracle.get()
    assert o.selfcheck(), "oracle build is not exact (FMA contraction or double rounding)"
    return o
