import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test")
    config.addinivalue_line("markers", "oracle_job(*names): compares against a long FP64 oracle run "
                                       "(tests/_oracle_refs.py), started in the background at collection")


def pytest_collection_finish(session):
    """Start the long oracle runs of the selected full-length GPU tests right away, in
    spawned processes, so that they overlap the rest of the GPU suite."""
    names = set()
    for item in session.items:
        m = item.get_closest_marker("oracle_job")
        if m is not None:
            names.update(m.args)
    if not names:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    import _oracle_refs
    _oracle_refs.start(sorted(names))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("_oracle_refs")
    if mod is not None:
        mod.stop()


@pytest.fixture(scope="session")
def lib():
    """The C-ABI library through its Python binding (builds it if needed)."""
    import paper_1808_06357_gb300 as lsp
    return lsp
