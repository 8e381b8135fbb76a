import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


# Modules collected after every other test, so that a failure in them (under -x) comes after the
# rest of the suite has run: the newest paths, whose GPU runs are the fewest.
_COLLECT_LAST = ("test_gpu_fch2d.py",)


def pytest_collection_modifyitems(session, config, items):
    # stable sort: the rest keep their order
    items.sort(key=lambda it: os.path.basename(it.nodeid.split("::")[0]) in _COLLECT_LAST)
