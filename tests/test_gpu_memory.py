"""Device memory of the library (needs a GB300): buffers come from a stream-ordered pool of the
library's own that keeps its reserve across contexts; gfcc_release_cached_memory gives it back."""
import numpy as np
import pytest

from gpu_util import inputs, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def test_contexts_on_two_streams_reuse_pool_memory(torch):
    """Two contexts on two streams, created, used and freed in turn (each reuses memory the other gave
    back to the pool): the same G as one context on the default stream; after the release call the
    device has at least as much free memory as before it."""
    from paper_1902_06016_gb300 import Context, gfcc
    inp = inputs(7, 13, 103)
    ws = np.linspace(-1.0, 0.0, 5)
    orb = list(range(7))
    ref = Context(inp, tol=1e-11)
    G0 = ref.solve_full(ws, 0.01, orb)["G"]
    ref.close()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for rnd in range(2):
        for st in (s1, s2):
            ctx = Context(inp, tol=1e-11, stream=st.cuda_stream)
            G = ctx.solve_full(ws, 0.01, orb)["G"]
            ctx.close()
            assert rel_err(G, G0) <= 1e-12, (rnd, st)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    gfcc.release_cached_memory()
    after = torch.cuda.mem_get_info()[0]
    assert after >= before
