import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long CPU test")
    config.addinivalue_line(
        "markers", "oracle_jobs(*jobs): full-size oracle runs started in the background when the session starts"
    )


def pytest_collection_finish(session):
    """Starts the oracle runs that the selected full-size parity tests need
    (spawned processes), so that they overlap the rest of the GPU tests."""
    jobs = []
    for item in session.items:
        for m in item.iter_markers("oracle_jobs"):
            jobs.extend(m.args)
    if not jobs:
        return
    try:
        import torch

        if not torch.cuda.is_available():
            return
    except Exception:
        return
    import oracle
    import oracle_jobs

    oracle.build()  # once, before the workers load it
    oracle_jobs.start(list(dict.fromkeys(jobs)))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.stop()
