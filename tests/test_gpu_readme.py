"""The Python example of the top-level README runs as written."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    from paper_2509_04955_gb300 import build as B
    B.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    assert abs(ns["state"].norm() - 1) < 1e-4
    assert ns["theta"].grad is not None and ns["theta"].grad.shape == ns["theta"].shape
