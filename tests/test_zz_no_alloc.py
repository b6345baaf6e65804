"""The allocation-free time step (glbe_step_residual_noalloc) against the
regular context path.

The allocation-free entry point exists for callers that cannot call
cudaMalloc (their device memory belongs to another allocator) and so cannot
hand the library a workspace.  It runs the same fused residual step on the
caller's own population and velocity buffers, with its scratch in a static
device array inside the library.  This test drives it call after call from the
rest state and checks every call's velocity output, and the residual of the
two evaluations (levels 10 and 20), against what a glbe_init context computes
for the same problem, within the per-step parity tolerance of the other GPU
tests.  The file is collected last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# per-step parity tolerance of each storage form (tests/test_gpu_parity.py)
TOL = {"f32": 3e-5, "f32c": 3e-5, "f16": 4e-3, "bf16": 3e-2}
BYTES = {"f32": 4, "f32c": 6, "f16": 2, "bf16": 2}


# x periodic with an even nx: the 16-bit forms run the paired kernel (two
# nodes per thread, its partials per 128-thread block); walls along x: every
# form runs the one-node kernel.  F32C exercises the compensated layout (high
# parts, then the FP16 low parts) in the caller's buffers.
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16", "f32c"])
@pytest.mark.parametrize("xwalls", [False, True])
def test_noalloc_step_matches_context_path(storage, xwalls):
    import torch
    from paper_0809_4730_gb300 import glbe
    from paper_0809_4730_gb300.inputs import duct_force_x
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    nx, ny, nz = 40, 22, 18
    N = nx * ny * nz
    w = int(xwalls)
    kw = dict(wall_lo=(w, 1, 1), wall_hi=(w, 1, 1), gamma=0.2, nu=0.02, force_field=1, storage=storage)
    ref = glbe.Solver(nx, ny, nz, **kw)
    Fx = torch.tensor(duct_force_x(nx, ny, nz, F0=2e-5)[0].reshape(1, -1), dtype=torch.float32, device="cuda")
    ref.set_force(Fx)

    p = ref.params                       # same parameters, same stream
    src = torch.zeros(19 * N * BYTES[storage], dtype=torch.uint8, device="cuda")    # rest state
    dst = torch.zeros_like(src)
    u_prev = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    u_tmp = torch.zeros_like(u_prev)

    def rel(a, b):
        b = b.double().cpu().numpy()
        a = a.double().cpu().numpy()
        s = np.abs(b).max()
        return np.abs(a - b).max() / (s if s > 0 else 1.0)

    tol = TOL[storage]
    compared = 0
    for t in range(0, 21):
        _, u_ref, _ = ref.fields()                 # u of level t from the context path
        at_level = (t % 10 == 0)
        u_out = u_prev if at_level else u_tmp
        info = glbe.glbe_step_residual_noalloc(p, src, dst, Fx, u_out, have_prev=at_level and t > 0, t=t)
        ref.step(1)
        torch.cuda.synchronize()
        assert rel(u_out, u_ref.reshape(-1)) <= tol, f"velocity of level {t}"
        if at_level and t > 0:
            want = ref.residual()
            assert want.t == t and info.t == t
            assert abs(info.r - want.r) <= max(1e-6, tol) * want.r
            assert abs(info.mass - want.mass) <= 1e-12 * want.mass
            assert info.nonfinite == 0
            compared += 1
        src, dst = dst, src
    assert compared == 2
    ref.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_0809_4730_gb300 import glbe
    import torch
    p = glbe.glbe_params_default()
    p.nx, p.ny, p.nz = 256, 256, 65        # 4,259,840 nodes > 4,194,304
    p.nu = 0.1
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(glbe.GlbeError) as ei:
        glbe.glbe_step_residual_noalloc(p, x, x[8:], None, x, False, 0)
    assert ei.value.status == glbe.GLBE_ERR_ARG
    # a buffer that is not 16-byte aligned is refused on the host
    p.nx, p.ny, p.nz = 4, 4, 4
    with pytest.raises(glbe.GlbeError) as ei:
        glbe.glbe_step_residual_noalloc(p, x[1:], x[8:], None, x, False, 0)
    assert ei.value.status == glbe.GLBE_ERR_ARG
