import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionfinish(session, exitstatus):
    """With EBR_PARITY_REPORT=<path>, write the worst errors the parity checks
    observed (per quantity: fraction of its tolerance, measured value) as JSON."""
    path = os.environ.get("EBR_PARITY_REPORT")
    if not path:
        return
    mod = sys.modules.get("tests.parity")
    if mod is None:
        return
    import json
    with open(path, "w") as fh:
        json.dump({k: {"of_tolerance": v[0], "value": v[1]} for k, v in sorted(mod.WORST.items())}, fh, indent=1)
