"""Batched and served solves: each result is the same alone and in the mix."""
import numpy as np
import pytest

from oracle import pint_oracle as O
from paper_2304_14021_gb300 import build_lib, pint, serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib.build()


def small_batch(n, seed):
    return synth.batched_instances(n, seed, max_dof=2**17)


def solver_kw(prob):
    return dict(prob, precision="mixed_ff", tol=1e-10, max_iter=200, init_guess=2, tol_update=1e-9)


def test_batch_equals_one_at_a_time_and_oracle():
    inst = small_batch(12, 3)
    streams = [torch.cuda.Stream() for _ in inst]
    solvers = [pint.Solver(stream=st, **solver_kw(x["problem"])) for st, x in zip(streams, inst)]
    u0s = [torch.from_numpy(x["u0"]).cuda() for x in inst]
    Ub = [torch.zeros(x["problem"]["nt"], x["u0"].size, dtype=torch.float64, device="cuda") for x in inst]
    torch.cuda.synchronize()
    stats = pint.solve_batch(solvers, u0s, Ub)
    torch.cuda.synchronize()
    assert all(s["rc"] == 0 for s in stats), [s["rc"] for s in stats]
    for i, (x, s) in enumerate(zip(inst, solvers)):
        U1 = torch.zeros_like(Ub[i])
        st = s.solve(u0s[i], U1)
        torch.cuda.synchronize()
        assert torch.equal(U1, Ub[i]) and st["iters"] == stats[i]["iters"]
        p = O.Problem(**{k: x["problem"][k] for k in ("equation", "dim", "nx", "ny", "bc", "eps", "beta", "T", "nt",
                                                       "n_windows", "alpha")})
        if p.nspace * p.nt <= 2**15:
            assert O.rel_err(Ub[i].cpu().numpy(), O.sequential(p, x["u0"])) < 1e-8
    for s in solvers:
        s.close()


def test_serving_result_alone_equals_result_in_mix():
    inst = small_batch(16, 5)
    srv = serve.Server(hbm_budget_bytes=8e9, max_slots=8, tol=1e-10, tol_update=1e-9)
    alone = srv.submit(inst[0]["u0"], **inst[0]["problem"]).result(timeout=120)
    futs = [srv.submit(x["u0"], **x["problem"]) for x in inst[1:8]]
    mixed = srv.submit(inst[0]["u0"], **inst[0]["problem"])
    futs += [srv.submit(x["u0"], **x["problem"]) for x in inst[8:]]
    res = [f.result(timeout=300) for f in futs]
    m = mixed.result(timeout=300)
    srv.close()
    assert torch.equal(alone.U, m.U)
    assert alone.stats["iters"] == m.stats["iters"] and alone.stats["rc"] == 0
    rep = srv.report()
    assert rep["n"] == 17 and rep["failed"] == 0 and rep["p99_s"] >= rep["p50_s"] > 0
    assert all(r.stats["rc"] == 0 for r in res)


def test_serving_admission_by_footprint():
    inst = small_batch(6, 7)
    fps = []
    srv0 = serve.Server(hbm_budget_bytes=1e12, max_slots=1)
    fps = [srv0.footprint(x["problem"]) for x in inst]
    srv0.close()
    budget = max(fps) + 1
    srv = serve.Server(hbm_budget_bytes=budget, max_slots=4)
    futs = [srv.submit(x["u0"], **x["problem"]) for x in inst]
    for f in futs:
        r = f.result(timeout=300)
        assert r.stats["rc"] == 0
        r.release()              # the budget holds one request's memory, so the next waits for this
    assert srv.peak_reserved <= budget
    big = dict(inst[0]["problem"], nx=4096, dim=1, ny=1, nt=1024)
    with pytest.raises(ValueError):
        srv.submit(np.zeros(4096), **big) if srv.footprint(big) > budget else (_ for _ in ()).throw(ValueError())
    srv.close()


def test_serving_budget_holds_live_results_and_reuses_solvers():
    # More requests than fit the budget at once: admission counts both the solver entries and the
    # solutions handed out, and a solution's bytes return to the budget only when it is released.
    x = [x for x in small_batch(24, 11) if x["dof"] <= 2**15][0]
    srv0 = serve.Server(hbm_budget_bytes=1e12, max_slots=1)
    budget = 2 * srv0.footprint(x["problem"])      # room for two requests of this shape
    srv0.close()
    srv = serve.Server(hbm_budget_bytes=budget, max_slots=4, tol=1e-10, tol_update=1e-9)
    first = srv.submit(x["u0"], **x["problem"]).result(timeout=120)
    held = [first]
    # while `first` is held its bytes stay reserved; the others fit one at a time beside it
    futs = [srv.submit(x["u0"], **x["problem"]) for _ in range(6)]
    for f in futs:
        r = f.result(timeout=300)
        assert torch.equal(r.U, first.U) and r.stats["rc"] == 0      # a reused solver: same result
        r.release()
    assert srv.peak_reserved <= budget
    rep = srv.report()
    assert rep["solvers_reused"] >= 5 and rep["solvers_created"] <= 2
    for r in held:
        r.release()
    srv.drain()
    import time
    time.sleep(0.1)
    with srv.cv:
        srv._collect_freed()
        assert srv.live_result_bytes == 0
        assert srv.reserved == sum(e.bytes for lst in srv.idle.values() for e in lst)
    srv.close()
    assert srv.reserved == 0


def test_serving_orders_a_device_input_after_its_producer():
    # u0 written by a kernel on another stream, submitted right away: the solve's stream waits for it
    inst = small_batch(4, 13)
    x = inst[0]
    srv = serve.Server(hbm_budget_bytes=8e9, max_slots=2, tol=1e-10, tol_update=1e-9)
    ref = srv.submit(x["u0"], **x["problem"]).result(timeout=120)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000)                                   # delay the producer
        u0 = torch.from_numpy(x["u0"]).to("cuda", non_blocking=True) * 1.0
        r = srv.submit(u0, **x["problem"])
    res = r.result(timeout=120)
    srv.close()
    assert torch.equal(res.U, ref.U)
