"""The stochastically rounded 16-bit storage forms (GLBE_BF16_SR,
GLBE_F16_SR) through the C-ABI.

In a fully periodic box under a uniform force from rest the state stays
uniform and every node's momentum is j(t) = (t + 1/2) F / gamma exactly (the
half-force of Eq. precondhydrofields and the conserved-row source F/gamma of
Eq. precondsourceterm).  Each step adds about w_a 3 e_a.F / gamma to the
populations; once that is below half a unit in the last place of a stored
BF16 value, round-to-nearest drops it at every node alike and j(t) stops
growing, while an unbiased stochastic rounding keeps the mean growth exact,
up to a zero-mean noise that averages out over the nodes.
"""
import numpy as np
import pytest

from gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def _box(storage, F=(1e-6, 0.0, 0.0), gamma=1.0, n=16, **kw):
    from paper_0809_4730_gb300.glbe import Solver
    require_cuda()
    return Solver(n, n, n, gamma=gamma, nu=0.1, F=F, storage=storage, **kw)


@pytest.mark.parametrize("storage,gamma", [("bf16sr", 1.0), ("f16sr", 1.0), ("bf16sr", 0.5)])
def test_uniform_forcing_momentum_is_unbiased(storage, gamma):
    F = np.array([1e-6, -5e-7, 0.0])
    G = _box(storage, F=tuple(F), gamma=gamma)
    N = 16 ** 3
    G.step(2001)                      # the record of level 2000
    info = G.residual()
    assert info.t == 2000
    want = N * (2000 + 0.5) * F / gamma
    got = np.array(info.momentum[:])
    # noise: about one unit in the last place per population and step,
    # independent between nodes; 1e-2 of the momentum is > 10 standard deviations
    assert np.abs(got - want).max() <= 1e-2 * np.abs(want).max(), (got, want)
    G.close()


def test_round_to_nearest_stagnates_where_stochastic_rounding_does_not():
    """The same march with BF16 round-to-nearest loses most of the momentum
    growth: the failure the stochastic forms exist to remove."""
    F = np.array([1e-6, 0.0, 0.0])
    N = 16 ** 3
    want = N * 2000.5 * F[0]
    G = _box("bf16", F=tuple(F))
    G.step(2001)
    rn = G.residual().momentum[0]
    G.close()
    assert rn < 0.8 * want, (rn, want)


@pytest.mark.parametrize("storage", ["bf16sr", "f16sr"])
def test_stochastic_rounding_is_reproducible(storage):
    """The random bits are counter-based (node, population, step seed): two
    contexts march bit for bit alike, and the march differs from
    round-to-nearest."""
    from paper_0809_4730_gb300.inputs import duct_force_x
    torch = require_cuda()
    kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.2, force_field=1)
    Fx = torch.tensor(duct_force_x(32, 18, 14, F0=1e-5)[0].reshape(1, -1), dtype=torch.float32, device="cuda")
    out = []
    for st in (storage, storage, storage.replace("sr", "")):
        from paper_0809_4730_gb300.glbe import Solver
        G = Solver(32, 18, 14, nu=0.05, storage=st, **kw)
        G.set_force(Fx)
        G.step(57)
        df, _, _ = G.get_state()
        G.sync()
        out.append(df.cpu().numpy())
        G.close()
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])


@pytest.mark.parametrize("storage", ["bf16sr", "f16sr"])
def test_stochastic_rounding_in_a_captured_solve_matches_steps(storage):
    """glbe_solve replays a captured 10-step chunk; the rounding seed lives
    in device memory, so the replayed chunks round exactly as glbe_step_n
    does."""
    from paper_0809_4730_gb300.glbe import GLBE_ERR_TIMEOUT, Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    torch = require_cuda()
    kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.2, force_field=1, nu=0.05, storage=storage)
    Fx = torch.tensor(duct_force_x(32, 18, 14, F0=1e-5)[0].reshape(1, -1), dtype=torch.float32, device="cuda")
    A = Solver(32, 18, 14, **kw)
    B = Solver(32, 18, 14, **kw)
    A.set_force(Fx)
    B.set_force(Fx)
    st, steps, r = A.solve(1e-30, 200)           # no convergence: 200 steps of replayed chunks
    assert st == GLBE_ERR_TIMEOUT and A.t == 200
    B.step(200)
    a, _, _ = A.get_state()
    b, _, _ = B.get_state()
    A.sync()
    assert torch.equal(a, b)
    A.close()
    B.close()
