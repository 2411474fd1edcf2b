import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def golden():
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def acuity():
    import oracle
    return oracle.Acuity()


@pytest.fixture(scope="session")
def layout(acuity):
    import oracle
    return oracle.lp_layout(acuity)


@pytest.fixture(scope="session")
def V():
    """The C-ABI binding, built in-tree (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_23410_gb300 import build
    build.build()
    from paper_2503_23410_gb300 import vafr
    vafr.load()
    torch.cuda.set_device(0)
    return vafr


@pytest.fixture(scope="session")
def torch_mod():
    import torch
    return torch


def pytest_terminal_summary(terminalreporter):
    """Widest classified ray-edge / depth tie of the session, per kind."""
    mod = sys.modules.get("parity")
    if not mod or not getattr(mod, "TIE_WIDTHS", None):
        return
    worst = {}
    for kind, w in mod.TIE_WIDTHS:
        n, m = worst.get(kind, (0, 0.0))
        worst[kind] = (n + 1, max(m, w))
    terminalreporter.write_line("classified ties (count, widest): " + ", ".join(
        f"{k} {n} {m:.3e}" for k, (n, m) in sorted(worst.items())))
