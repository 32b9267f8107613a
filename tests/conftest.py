import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "late(rank=1): run after every other test (see pytest_collection_modifyitems)")
    spec = os.environ.get("ORACLE_MUTANT")
    if spec:
        _plant_oracle_mutant(spec)


def pytest_collection_modifyitems(config, items):
    """Tests marked late run after all the others, ordered by the marker's
    rank (late(2) after late) and otherwise as collected: under -x a failure
    there leaves every other test already run."""
    def rank(it):
        m = it.get_closest_marker("late")
        return 0 if m is None else (m.args[0] if m.args else 1)

    items.sort(key=rank)


def _plant_oracle_mutant(spec):
    """Swap one oracle module's functions and constants for those of a copy of
    its source with one textual change planted in it. Only the child pytest
    processes of test_oracle_mutants.py set ORACLE_MUTANT; the oracle files
    themselves are never modified."""
    import importlib
    import inspect
    import json

    s = json.loads(spec)
    mod = importlib.import_module(s["module"])
    src = inspect.getsource(mod)
    if src.count(s["old"]) != 1:
        raise pytest.UsageError(f"mutation target occurs {src.count(s['old'])} times in {s['module']}")
    ns = {"__name__": mod.__name__, "__package__": mod.__package__, "__spec__": mod.__spec__,
          "__file__": mod.__file__}
    exec(compile(src.replace(s["old"], s["new"]), mod.__file__, "exec"), ns)
    for k, v in ns.items():
        if not k.startswith("__"):
            setattr(mod, k, v)
