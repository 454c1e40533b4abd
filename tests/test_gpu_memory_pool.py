"""The library's device memory pool: a context set up after another was
destroyed reuses the pool's blocks, rte_trim_memory returns the unused ones,
and results do not depend on whether a block came fresh or reused (the set-up
writes or clears everything it reads: D and the node tables are written whole,
the rest is zeroed)."""
import numpy as np
import pytest

from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _apply_once(md, x):
    from paper_2604_23265_gb300 import rte
    ctx = rte.Context.from_medium(md)
    y = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.apply(x, y)
    z = torch.zeros(ctx.n, dtype=torch.float32, device="cuda")
    ctx.block_apply(x.float(), z)
    torch.cuda.synchronize()
    out = (y.cpu().numpy(), z.cpu().numpy())
    ctx.close()
    return out


def test_reused_and_trimmed_pool_give_identical_results(lib):
    from paper_2604_23265_gb300 import rte
    md = W.grf_diffusive(seed=3, I=48, M=16)
    n = 2 * md.M * md.I * md.I
    x = torch.tensor(W.random_vector(n, 7), device="cuda")
    first = _apply_once(md, x)
    # a larger context in between leaves other contents in the pool's blocks
    big = rte.Context.from_medium(W.grf_diffusive(seed=4, I=64, M=16))
    big.close()
    reused = _apply_once(md, x)
    rte.trim_memory()
    fresh = _apply_once(md, x)
    for a, b, c in zip(first, reused, fresh):
        assert np.array_equal(a, b) and np.array_equal(a, c)
