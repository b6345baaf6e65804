"""Checkpoint / resume through the C-ABI (glbe_checkpoint_*): a march that
is saved, continued, restored into a fresh context and continued again must
reproduce the first continuation bit for bit, including the compensated
storage's low parts, the coupled lattice, the force field and the residual
levels."""
import numpy as np
import pytest

from gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def _solver(storage, mhd, variant=0):
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import random_force
    torch = require_cuda()
    kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 0), gamma=0.3, nu=0.03, storage=storage, force_field=3,
              variant=variant)
    if mhd:
        kw.update(induction=1, gamma_m=0.3, eta=0.03, chi=0.2, mu=1.0, B0=(0.0, 0.02, 0.0))
    G = Solver(24, 10, 9, **kw)
    F = random_force(24, 10, 9, 2e-5, seed=3)
    G.set_force(torch.tensor(F.reshape(3, -1), dtype=torch.float32, device="cuda"))
    return G


def _state(G):
    G.sync()
    return [None if a is None else a.cpu().numpy() for a in G.get_state()]


# the stochastically rounded forms resume with the rounding seed of the saved level
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16", "f32c", "bf16sr", "f16sr"])
@pytest.mark.parametrize("mhd", [False, True])
def test_resume_is_bit_exact(storage, mhd):
    A = _solver(storage, mhd)
    A.step(37)                       # odd level, mid-way between residual levels
    ck = A.checkpoint()
    A.step(45)
    ra = A.residual()
    sa = _state(A)

    B = _solver(storage, mhd)
    B.restore(ck)
    assert B.t == 37
    B.step(45)
    rb = B.residual()
    sb = _state(B)
    assert rb.t == ra.t == 80
    assert rb.r == ra.r and rb.mass == ra.mass
    for a, b in zip(sa, sb):
        if a is not None:
            assert np.array_equal(a, b)
    # the raw states, low parts included, are byte-identical
    assert A.checkpoint() == B.checkpoint()


def test_checkpoint_of_another_shape_is_rejected():
    from paper_0809_4730_gb300.glbe import GLBE_ERR_ARG, GlbeError
    A = _solver("f32", False)
    ck = A.checkpoint()
    B = _solver("bf16", False)
    with pytest.raises(GlbeError) as ei:
        B.restore(ck)
    assert ei.value.status == GLBE_ERR_ARG
    with pytest.raises(GlbeError) as ei:
        A.restore(ck[: len(ck) // 2])
    assert ei.value.status == GLBE_ERR_ARG
    bad = bytearray(ck)
    bad[0:8] = b"NOTACKPT"
    with pytest.raises(GlbeError):
        A.restore(bytes(bad))
