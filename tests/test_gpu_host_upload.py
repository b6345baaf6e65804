"""Host force uploads through the C-ABI (glbe_set_force_host).

The upload is staged on the library's copy stream and overlaps the steps
already enqueued; the field must still apply exactly to the steps enqueued
after the call.  So a march whose force changes between steps must be bit for
bit the same whether the fields come from device memory (glbe_set_force) or
from pinned host memory, with the upload issued while earlier steps are still
running, and with two uploads in a row (the second waits for the first
hand-over)."""
import numpy as np
import pytest

from gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def _solver(storage):
    from paper_0809_4730_gb300.glbe import Solver
    return Solver(32, 12, 10, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.3, nu=0.03, storage=storage,
                  force_field=3)


def _fields(torch, seeds):
    from paper_0809_4730_gb300.inputs import random_force
    return [torch.tensor(random_force(32, 12, 10, 3e-5, seed=s).reshape(3, -1), dtype=torch.float32) for s in seeds]


def _state(G):
    G.sync()
    return [None if a is None else a.cpu().numpy() for a in G.get_state()]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_host_upload_matches_device_upload(storage):
    torch = require_cuda()
    from paper_0809_4730_gb300.glbe import glbe_set_force_host
    F1, F2, F3 = _fields(torch, (1, 2, 3))

    A = _solver(storage)
    A.set_force(F1.cuda())
    A.step(23)
    A.set_force(F2.cuda())
    A.step(17)
    A.set_force(F3.cuda())
    A.step(9)
    ra = A.residual()
    sa = _state(A)

    B = _solver(storage)
    h1, h2, h3 = (F.pin_memory() for F in (F1, F2, F3))
    glbe_set_force_host(B.ctx, h1)
    B.step(23)
    glbe_set_force_host(B.ctx, h2)     # overlaps the 23 steps in flight
    B.step(17)
    glbe_set_force_host(B.ctx, h1)     # two uploads in a row: the last one applies
    glbe_set_force_host(B.ctx, h3)
    B.step(9)
    rb = B.residual()
    sb = _state(B)
    assert rb.t == ra.t and rb.r == ra.r and rb.mass == ra.mass
    for a, b in zip(sa, sb):
        if a is not None:
            assert np.array_equal(a, b)
