"""The README's quick-start example runs as written (the Python block of its
"Quick start" section), and its result agrees with the library's own calls."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_quick_start_runs():
    import torch
    text = open(os.path.join(ROOT, "README.md")).read()
    section = text[text.index("## Quick start"):]
    code = re.search(r"```python\n(.*?)```", section, flags=re.S).group(1)
    env = {}
    exec(compile(code, "README.md", "exec"), env)  # noqa: S102 - the repository's own documentation
    res, cost, argmin, solver = env["res"], env["cost"], env["argmin"], env["solver"]
    torch.cuda.synchronize()
    B = env["sc"].goals.shape[0]
    assert res.coef.shape == (B, 3 * solver.n) and cost.shape == (B,)
    assert torch.isfinite(res.coef).all()
    assert 0 <= int(argmin.item()) < B
    assert float(cost[int(argmin.item())]) == float(cost.min())
    solver.status()
    solver.close()
