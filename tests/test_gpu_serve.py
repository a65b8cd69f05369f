"""The served batch (continuous batching of mixed-precision solves).

* A request's result is the same alone and in a mix whose membership changes
  while it runs (requests admitted and retired around it): bitwise, because
  a request's arithmetic does not depend on the others; the bar asked of the
  mixed path (1e-8 relative) is asserted as well.
* Served results match the FP64 oracle to 1e-8, also in a mix that takes
  every path of the preconditioner items at once: staged by bulk tensor
  copies (with a box deeper than the grid), read directly (rows that are not
  16-byte multiples) and one thread per column (more than 128 levels).
* Admission respects the device-byte budget; a request larger than the budget
  is refused at submission; a request with a non-finite right-hand side ends
  in breakdown without disturbing the others.
* The multigrid mode (FP64 CG with the FP32 V-cycle, a worker pool) matches
  the oracle, gives a request the same result alone and in a mix, keeps more
  than one solve in flight and respects the budget.
"""
import numpy as np
import pytest

import workloads as W
from oracle import FluxOperator, LinePreconditioner, assemble_csr, pcg_interleaved

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need cuda:0"
    import paper_1302_7193_gb300 as pkg
    from paper_1302_7193_gb300 import build as B
    B.build()
    return pkg


def _mix():
    reqs = W.request_stream(duration_s=1.0, rate_hz=50.0, seed=7, sizes=(16, 32, 48), levels=(8, 16, 32),
                            max_requests=8)
    return [(r.problem, W.rhs_for(r.problem, seed=r.rhs_seed)) for r in reqs]


def _drain(srv, ids, max_steps=100000):
    out = {}
    for _ in range(max_steps):
        for i in list(ids):
            got = srv.poll(i)
            if got is not None:
                out[i] = got
                ids.remove(i)
        if not ids:
            return out
        srv.step(8)
    raise AssertionError("served requests did not finish")


def test_alone_equals_in_mix(pkg):
    mix = _mix()
    probe = 3
    p, b = mix[probe]
    with pkg.Server(budget_bytes=1 << 30, max_slots=4) as srv:
        rid = srv.submit(p, b, tol=1e-10)
        alone = _drain(srv, [rid])[rid]
    with pkg.Server(budget_bytes=1 << 30, max_slots=4) as srv:
        ids = [srv.submit(q, bq, tol=1e-10) for q, bq in mix[:5]]       # probe is the fourth of five
        srv.step(8)
        ids += [srv.submit(q, bq, tol=1e-10) for q, bq in mix[5:]]      # arrive while the others run
        res = _drain(srv, list(ids))
    x_mix, st_mix = res[ids[probe]]
    x_alone, st_alone = alone
    assert st_mix.status == st_alone.status == 0
    assert st_mix.iterations == st_alone.iterations and st_mix.outer_sweeps == st_alone.outer_sweeps
    assert np.linalg.norm(x_mix - x_alone) <= 1e-8 * np.linalg.norm(x_alone)
    assert np.array_equal(x_mix, x_alone)


def test_served_results_match_oracle(pkg):
    mix = _mix()[:4]
    with pkg.Server(budget_bytes=1 << 30, max_slots=8) as srv:
        ids = [srv.submit(q, bq, tol=1e-10) for q, bq in mix]
        res = _drain(srv, list(ids))
    for (p, b), rid in zip(mix, ids):
        x, st = res[rid]
        assert st.status == 0
        ref = pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
        assert np.linalg.norm(x - ref.x.ravel()) / np.linalg.norm(ref.x) < 1e-8


def test_budget_bounds_admission(pkg):
    p = W.box_problem(64, 64, 32, 0.01, lambda2=0.1)
    per = 36 * p.n_cells + 2 * 8 * (3 * 32 + 64 + 2 * 64 * 64 + 2 * 32) + 16 * 1024
    with pkg.Server(budget_bytes=int(2.5 * per), max_slots=16) as srv:
        ids = [srv.submit(p, W.rhs_for(p, seed=s), tol=1e-8) for s in range(5)]
        peak = 0
        out = {}
        for _ in range(100000):
            for i in list(ids):
                got = srv.poll(i, want_x=False)
                if got is not None:
                    out[i] = got
                    ids.remove(i)
            if not ids:
                break
            active, pending = srv.step(4)
            peak = max(peak, active)
            assert srv.info()["used_bytes"] <= 2.5 * per
        assert not ids and peak == 2
        assert all(st.status == 0 for _, st in out.values())


def test_oversize_and_bad_requests(pkg):
    small = W.box_problem(16, 16, 8, 0.01)
    with pkg.Server(budget_bytes=64 << 20, max_slots=4) as srv:
        big = W.box_problem(512, 512, 64, 0.01)
        with pytest.raises(pkg.PCGError) as e:
            srv.submit(big, np.zeros(big.n_cells))
        assert e.value.code == pkg.PCG_ERR_OOM
        bad = W.rhs_for(small, seed=1)
        bad.ravel()[17] = np.nan
        good_id = srv.submit(small, W.rhs_for(small, seed=2), tol=1e-8)
        bad_id = srv.submit(small, bad, tol=1e-8)
        res = _drain(srv, [good_id, bad_id])
    assert res[good_id][1].status == 0
    assert res[bad_id][1].status == pkg.PCG_BREAKDOWN


def test_every_preconditioner_path_in_one_mix(pkg):
    probs = [W.box_problem(18, 10, 12, 0.01, name="rows-not-16B"),
             W.box_problem(8, 8, 160, 0.01, name="column-mode"),
             W.box_problem(40, 24, 40, 0.01, alpha="sin", name="staged-deep-box"),
             W.latlon_problem(36, 16, 24, name="latlon-staged")]
    mix = [(p, W.rhs_for(p, seed=i + 3)) for i, p in enumerate(probs)]
    with pkg.Server(budget_bytes=1 << 30, max_slots=8) as srv:
        ids = [srv.submit(q, bq, tol=1e-10) for q, bq in mix]
        res = _drain(srv, list(ids))
    for (p, b), rid in zip(mix, ids):
        x, st = res[rid]
        assert st.status == 0, (p.name, st)
        ref = pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
        assert np.linalg.norm(x - ref.x.ravel()) / np.linalg.norm(ref.x) < 1e-8, p.name
    for k in (0, 1, 2):
        with pkg.Server(budget_bytes=1 << 30, max_slots=8) as srv:
            rid = srv.submit(*mix[k], tol=1e-10)
            x_alone, st_alone = _drain(srv, [rid])[rid]
        assert np.array_equal(x_alone, res[ids[k]][0]), probs[k].name


# ---------------------------------------------------------------------------
# Multigrid mode: each request solved by FP64 CG with the FP32 V-cycle, by a
# pool of worker threads with a stream each.
# ---------------------------------------------------------------------------

def _mg_bytes(p):
    return 96 * p.n_cells + (1 << 20)


def test_multigrid_server_matches_oracle_and_alone(pkg):
    # tol 1e-12 as the oracle's: at the mix's strongest anisotropy a stop at 1e-10
    # leaves the near-constant mode about 1e-8 off
    mix = _mix()
    with pkg.Server(budget_bytes=1 << 30, max_slots=8, preconditioner="multigrid-f32") as srv:
        ids = [srv.submit(q, bq, tol=1e-12) for q, bq in mix[:5]]
        srv.step(8)
        ids += [srv.submit(q, bq, tol=1e-12) for q, bq in mix[5:]]      # arrive while the others run
        res = _drain(srv, list(ids))
    for (p, b), rid in list(zip(mix, ids))[:4]:
        x, st = res[rid]
        assert st.status == 0 and 0 < st.iterations < 200, st
        ref = pcg_interleaved(FluxOperator(p), LinePreconditioner(assemble_csr(p), p), b, eps=1e-12, maxiter=20000)
        err = np.linalg.norm(x - ref.x.ravel()) / np.linalg.norm(ref.x)
        assert err < 1e-8, (p.name, err)
    probe = 3
    with pkg.Server(budget_bytes=1 << 30, max_slots=1, preconditioner="multigrid-f32") as srv:
        rid = srv.submit(*mix[probe], tol=1e-12)
        x_alone, st_alone = _drain(srv, [rid])[rid]
    assert st_alone.iterations == res[ids[probe]][1].iterations
    assert np.array_equal(x_alone, res[ids[probe]][0])


def test_multigrid_server_overlaps_and_bounds_admission(pkg):
    p = W.box_problem(128, 128, 64, 0.002, lambda2=0.01)
    per = _mg_bytes(p)
    with pkg.Server(budget_bytes=int(2.5 * per), max_slots=16, preconditioner="multigrid-f32") as srv:
        ids = [srv.submit(p, W.rhs_for(p, seed=s), tol=1e-8) for s in range(6)]
        peak, out = 0, {}
        for _ in range(100000):
            for i in list(ids):
                got = srv.poll(i, want_x=False)
                if got is not None:
                    out[i] = got
                    ids.remove(i)
            if not ids:
                break
            active, pending = srv.step(4)
            peak = max(peak, active)
            assert srv.info()["used_bytes"] <= 2.5 * per
        assert not ids and peak == 2              # two solves in flight at once, never three
        assert all(st.status == 0 for _, st in out.values())
        # restarted until the true residual meets tol or twice its FP64 rounding floor
        assert all(st.relres_true < 1e-8 or st.relres_true <= 2.0 * st.relres_floor for _, st in out.values())


def test_multigrid_server_refuses_oversize_and_other_preconditioners(pkg):
    with pkg.Server(budget_bytes=64 << 20, max_slots=4, preconditioner="multigrid-f32") as srv:
        big = W.box_problem(256, 256, 64, 0.01)
        with pytest.raises(pkg.PCGError) as e:
            srv.submit(big, np.zeros(big.n_cells))
        assert e.value.code == pkg.PCG_ERR_OOM
    import ctypes
    lib = pkg.load_library()
    o = pkg.pcg_opts_t(pkg.PCG_MIXED, 0.0, 0, 0, 0, ctypes.c_void_p(0), pkg.PCG_PREC_MULTIGRID)
    h = ctypes.c_void_p()
    rc = lib.pcg_server_create(ctypes.c_size_t(1 << 30), 4, ctypes.byref(o), ctypes.byref(h))
    assert rc == pkg.PCG_ERR_INVALID_ARG and not h.value
