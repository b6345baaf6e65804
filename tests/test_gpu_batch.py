"""Batched steady solves in one persistent launch (glbe_batch_*) against the
single-context path.

Both paths apply the same one-node-per-thread update to the same states, so
every domain of a batch must converge at the same residual level as its own
context and end with the same fields; the residual sums are reduced in a
different order (per tile vs per block), which may move a crossing by one
evaluation at most.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# (nx, ny, nz, gamma, Ha): odd and even sizes, flow-only and coupled domains
SPECS = [(12, 14, 10, 1.0, 0), (9, 16, 12, 0.1, 5), (16, 12, 12, 0.3, 0), (10, 18, 8, 0.1, 10), (7, 10, 10, 0.5, 5)]
# Ha = 20 at gamma = 0.1 on this grid is unstable (the FP64 oracle diverges too)
UNSTABLE = (10, 18, 8, 0.1, 20)


def _params(storage="f32", specs=SPECS):
    out = []
    for nx, ny, nz, gamma, Ha in specs:
        nu = eta = 0.02
        kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, F=(1e-5, 0, 0), storage=storage)
        if Ha > 0:
            L = (ny - 2) / 2
            kw.update(induction=1, gamma_m=gamma, eta=eta, chi=0.1, mu=1.0, B0=(0, Ha * math.sqrt(nu * eta) / L, 0))
        out.append((nx, ny, nz, kw))
    return out


def _batch(storage="f32", specs=SPECS):
    from paper_0809_4730_gb300.glbe import Batch, make_params
    return Batch([make_params(nx, ny, nz, **kw) for nx, ny, nz, kw in _params(storage, specs)])


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("storage", ["f32", "f32c"])
def test_batch_matches_single_contexts(storage):
    from paper_0809_4730_gb300.glbe import Solver
    tol = 1e-6
    B = _batch(storage)
    st, res, sec = B.solve(tol, 400_000, use_graph=True)
    assert st == 0, res
    assert sec > 0
    for d, (nx, ny, nz, kw) in enumerate(_params(storage)):
        G = Solver(nx, ny, nz, **kw)
        st2, steps2, r2 = G.solve(tol, 400_000)
        assert st2 == 0
        assert res[d]["converged"] and abs(res[d]["steps"] - steps2) <= 10, (d, res[d], steps2)
        assert 0 < res[d]["seconds"] <= sec
        if res[d]["steps"] == steps2:
            _, u_b, B_b = B.fields(d)
            _, u_s, B_s = G.fields()
            G.sync()
            assert _rel(u_b, u_s) <= 1e-6, d
            if B_b is not None:
                assert _rel(B_b, B_s) <= 1e-6, d
        G.close()
    B.close()


def test_batch_graph_and_direct_launch_agree():
    B = _batch()
    st1, r1, _ = B.solve(1e-6, 400_000, use_graph=True)
    B.reset()
    st2, r2, _ = B.solve(1e-6, 400_000, use_graph=False)
    assert st1 == st2 == 0
    assert [x["steps"] for x in r1] == [x["steps"] for x in r2]
    assert [x["r"] for x in r1] == [x["r"] for x in r2]
    B.close()


def test_batch_autotune_then_solve():
    B = _batch()
    st0, ref, _ = B.solve(1e-6, 400_000)
    B.reset()
    bt, bps, sps = B.autotune(12)
    assert bt in (128, 256) and bps >= 1 and sps > 0
    st, res, _ = B.solve(1e-6, 400_000)
    assert st0 == st == 0
    for a, b in zip(ref, res):
        assert abs(a["steps"] - b["steps"]) <= 10
    B.close()


def test_batch_solves_once_until_reset():
    from paper_0809_4730_gb300.glbe import GLBE_ERR_STATE, GlbeError
    B = _batch()
    st, _, _ = B.solve(1e-5, 400_000)
    assert st == 0
    with pytest.raises(GlbeError) as ei:
        B.solve(1e-5, 10)
    assert ei.value.status == GLBE_ERR_STATE
    B.reset()
    st, _, _ = B.solve(1e-5, 400_000)
    assert st == 0
    B.close()


def test_batch_barrier_wait_gives_up_and_the_batch_stays_usable():
    """One block leaves the launch at once (a flag nothing else sets), so the
    others' first grid-barrier wait runs to its poll limit; the launch must
    end with GLBE_ERR_TIMEOUT, not hang, and the batch must solve afterwards."""
    from paper_0809_4730_gb300.glbe import GLBE_ERR_TIMEOUT
    B = _batch()
    B.set_barrier_test(1 << 14, 0)
    st, res, _ = B.solve(1e-6, 1000)
    assert st == GLBE_ERR_TIMEOUT
    B.set_barrier_test(1 << 26, -1)
    B.reset()
    st, res, _ = B.solve(1e-6, 400_000)
    assert st == 0 and all(r["converged"] for r in res)
    B.close()


def test_batch_reports_the_unstable_domain_and_finishes_the_others():
    from paper_0809_4730_gb300.glbe import GLBE_ERR_DIVERGED
    specs = SPECS[:3] + [UNSTABLE]
    B = _batch(specs=specs)
    st, res, _ = B.solve(1e-6, 400_000)
    assert st == GLBE_ERR_DIVERGED
    assert res[3]["nonfinite"] and not res[3]["converged"]
    assert all(r["converged"] and not r["nonfinite"] for r in res[:3])
    B.close()


# ---------------------------------------------------------------------------
# The batch against the FP64 oracle itself.
# ---------------------------------------------------------------------------
def _oracle_cfg(orc, nx, ny, nz, kw):
    c = dict(wall_lo=kw["wall_lo"], wall_hi=kw["wall_hi"], gamma=kw["gamma"], nu=kw["nu"], F=kw["F"])
    if kw.get("induction"):
        c.update(induction=True, gamma_m=kw["gamma_m"], eta=kw["eta"], chi=kw["chi"], mu=kw["mu"], B0=kw["B0"])
    return orc.Config(nx, ny, nz, **c)


@pytest.mark.parametrize("storage", ["f32", "f32c"])
def test_batch_domains_match_oracle_after_23_levels(orc, storage):
    """Every domain (flow and coupled, gamma 1 to 0.1, odd and even sizes) is
    marched 23 levels from rest in one launch and compared node by node with
    the oracle's march of the same domain: the per-step parity bar of the
    single-context tests (3e-5 of the largest value)."""
    B = _batch(storage)
    st, res, _ = B.solve(1e-300, 23, use_graph=True)    # no domain leaves early
    from paper_0809_4730_gb300.glbe import GLBE_ERR_TIMEOUT
    assert st == GLBE_ERR_TIMEOUT and not any(r["converged"] for r in res)
    for d, (nx, ny, nz, kw) in enumerate(_params(storage)):
        S = orc.Solver(_oracle_cfg(orc, nx, ny, nz, kw))
        S.run(23)
        orho, ou, oB, _ = S.fields()
        fluid = ~S.solid_mask()
        rho, u, Bf = B.fields(d)
        torch_sync()
        u = u.double().cpu().numpy()[:, fluid]
        want = ou.T[:, fluid]
        assert np.abs(u - want).max() <= 3e-5 * np.abs(want).max(), d
        drho = rho.double().cpu().numpy()[fluid] - kw.get("rho0", 1.0)
        odr = orho[fluid] - 1.0
        assert np.abs(drho - odr).max() <= 3e-5 * np.abs(odr).max() + 2 ** -24, d
        if Bf is not None:
            b = Bf.double().cpu().numpy()[:, fluid] - np.asarray(kw["B0"])[:, None]
            ob = oB.T[:, fluid] - np.asarray(kw["B0"])[:, None]
            assert np.abs(b - ob).max() <= 3e-5 * np.abs(ob).max() + 2 ** -24 * np.abs(kw["B0"]).max(), d
    B.close()


def test_batch_steady_state_matches_converged_oracle(orc):
    """The batch solved to r <= 1e-8 (compensated storage) against the FP64
    oracle converged to 1e-11.  The ducts are x-periodic with walls in y and
    z and a uniform force, so their steady state is x-invariant and the
    oracle solves the 1 x ny x nz column.  Bar: the FP32 steady bar, velocity
    L-infinity relative error 1e-5."""
    B = _batch("f32c")
    st, res, _ = B.solve(1e-8, 400_000, use_graph=True)
    assert st == 0, res
    for d, (nx, ny, nz, kw) in enumerate(_params("f32c")):
        S = orc.Solver(_oracle_cfg(orc, 1, ny, nz, kw))
        S.run(3_000_000, tol=1e-11)
        _, ou, oB, _ = S.fields()
        col = ou[:, 0].reshape(nz, ny)
        _, u, Bf = B.fields(d)
        torch_sync()
        ux = u[0].double().cpu().numpy().reshape(nz, ny, nx)
        fl = (slice(1, nz - 1), slice(1, ny - 1))
        err = np.abs(ux[fl[0], fl[1], :] - col[fl][:, :, None]).max() / np.abs(col[fl]).max()
        assert err <= 1e-5, (d, err, res[d])
        if Bf is not None:
            bcol = oB[:, 0].reshape(nz, ny)
            bx = Bf[0].double().cpu().numpy().reshape(nz, ny, nx)
            eb = np.abs(bx[fl[0], fl[1], :] - bcol[fl][:, :, None]).max() / np.abs(bcol[fl]).max()
            assert eb <= 1e-4, (d, eb)
    B.close()


def torch_sync():
    import torch
    torch.cuda.synchronize()
