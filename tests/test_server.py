"""Continuous batching (hgks_server_*, hgks_batch_add/remove): solves that join
and leave a running batch give what they give alone.

A solve in the server follows Algorithm 1 exactly as alone (same parameters,
same kernels); only the summation order of its inner products differs, so the
steady state must agree with hgks_solve_steady's to the steady-state tolerance
(relative L2 1e-9) with the same number of steps, whatever else ran beside it
and whenever it was admitted.
"""
import time

import numpy as np
import pytest

import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REQUESTS = [
    ("sphere4", lambda: (I.sphere_mesh(4, 4, stretch=1.3), I.sphere_conditions(0.3, aoa_deg=4.0))),
    ("cavity3", lambda: (I.cavity_mesh(3, seed=I.BASE_SEED + 21), I.cavity_conditions(0.2, 80.0))),
    ("periodic4", lambda: (I.periodic_cube_mesh(4), I.sphere_conditions(0.35))),
    ("sphere3", lambda: (I.sphere_mesh(3, 6, stretch=1.25), I.sphere_conditions(0.45, aoa_deg=8.0))),
    ("cavity4", lambda: (I.cavity_mesh(4, seed=I.BASE_SEED + 22), I.cavity_conditions(0.3, 300.0))),
]
KW = dict(scheme=0, krylov_dim=8, restarts=2, jacobi_sweeps=2)
DROP, MAX_STEPS = 0.2, 25


def problems():
    out = []
    for k, (name, make) in enumerate(REQUESTS):
        m, cond = make()
        u = cond["u_inf"]
        base = (cond["rho_inf"], u[0] + 0.04, u[1] + 0.02, u[2] - 0.01, cond["p_inf"])
        Q0, _ = I.smooth_state(m, seed=I.BASE_SEED + 60 + k, amp=0.03, base=base)
        p = H.hgks_default_params(**{**cond, "Pr": 0.72 if cond["viscous"] else 1.0, **KW})
        out.append((name, m, cond, p, Q0))
    return out


def alone(m, p, Q0):
    import torch
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Qd = hm.to_internal(Q0)
    info, hist, conv = H.hgks_solve_steady(hm, p, Qd, None, drop_tol=DROP, max_steps=MAX_STEPS)
    torch.cuda.synchronize()
    return hm.to_caller(Qd), info


def test_server_results_equal_alone_with_memory_admission(cuda):
    probs = problems()
    largest = max(m.n_tet for _, m, _, _, _ in probs)
    shared = H.hgks_default_params(**KW)
    # an arena for about one and a half of the largest meshes: later requests wait for memory
    srv = H.hgks_server(shared, hbm_budget_bytes=int(1.6 * largest * 9000), max_inflight=8)
    cap = srv.info().n_cells
    assert largest <= cap < 3 * largest
    ids = {}
    for name, m, cond, p, Q0 in probs[:3]:
        ids[name] = srv.submit(m, p, Q0, drop_tol=DROP, max_steps=MAX_STEPS)
    waited_for_memory = False
    late = probs[3:]
    rounds = 0
    while True:
        fin, run, wait = srv.step()
        rounds += 1
        states = {n: srv.status(i).state for n, i in ids.items()}
        running = [n for n, s in states.items() if s == 2]
        # the running solves fit in the arena; a built request (state 1) waits only for room
        assert sum((m.n_tet + 255) // 256 * 256 for n, m, *_ in probs if n in running) <= cap
        if running and any(s == 1 for s in states.values()):
            waited_for_memory = True
        if rounds == 3:                          # more requests arrive while others run
            for name, m, cond, p, Q0 in late:
                ids[name] = srv.submit(m, p, Q0, drop_tol=DROP, max_steps=MAX_STEPS)
        if rounds > 3 and run == 0 and wait == 0:
            break
        if run == 0:
            time.sleep(0.005)                    # builds still running on the host
        assert rounds < 5000
    assert waited_for_memory
    for name, m, cond, p, Q0 in probs:
        st = srv.status(ids[name])
        assert st.state == 3, name
        Qs, _ = srv.collect(ids[name])
        Qa, ia = alone(m, p, Q0)
        assert st.solve.steps == ia.steps, f"{name}: {st.solve.steps} steps served, {ia.steps} alone"
        assert bool(st.solve.converged) == bool(ia.converged)
        rel = np.linalg.norm(Qs - Qa) / np.linalg.norm(Qa)
        assert rel <= 1e-9, f"{name}: served vs alone {rel:.3e}"
        assert st.t_submit <= st.t_built <= st.t_admit <= st.t_done


def test_batch_add_remove_reuses_ranges(cuda):
    import torch
    probs = problems()
    # A (384 tets) and B (384) fill the arena exactly; C (162) fits only into A's range once A leaves
    (_, mA, _, pA, QA), (_, mB, _, pB, QB), (_, mC, _, pC, QC) = probs[4], probs[2], probs[1]
    hA, hB, hC = (H.hgks_mesh_create(m, scheme_mask=1) for m in (mA, mB, mC))
    pad = lambda n: (n + 255) // 256 * 256
    assert pad(mC.n_tet) <= pad(mA.n_tet)
    cells = pad(mA.n_tet) + pad(mB.n_tet)
    b = H.hgks_batch_create_empty(cells, 3 * cells, 2, H.hgks_default_params(**KW))
    kA = H.hgks_batch_add(b, hA, pA)
    kB = H.hgks_batch_add(b, hB, pB)
    with pytest.raises(H.HGKSError):            # no free slot
        H.hgks_batch_add(b, hC, pC)
    H.hgks_batch_remove(b, kA)
    kC = H.hgks_batch_add(b, hC, pC)            # into the freed slot and range
    for k, hm, Q in ((kB, hB, QB), (kC, hC, QC)):
        H.hgks_batch_set_state(b, k, hm.to_internal(Q))
    H.hgks_batch_gmres_step(b)
    for k, hm, p, Q in ((kB, hB, pB, QB), (kC, hC, pC, QC)):
        Qd = hm.to_internal(Q)
        Q0 = Qd.clone()
        H.hgks_gmres_step(hm, p, Qd, None)
        Qb = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, k, Q=Qb)
        torch.cuda.synchronize()
        rel = (torch.linalg.norm((Qb - Q0) - (Qd - Q0)) / torch.linalg.norm(Qd - Q0)).item()
        assert rel <= 1e-10, rel
    assert H.hgks_batch_info(b).n_meshes == 2


def test_server_reports_a_failed_build(cuda):
    shared = H.hgks_default_params(**KW)
    srv = H.hgks_server(shared, hbm_budget_bytes=1 << 30, max_inflight=2)
    m, cond = I.cavity_mesh(2), I.cavity_conditions()
    bad = I.Mesh(m.xyz.copy(), m.tet4.copy(), m.bface3.copy(), m.btag.copy(), None)
    bad.xyz[:] = 0.0                              # every tetrahedron degenerate
    p = H.hgks_default_params(**{**cond, **KW})
    rid = srv.submit(bad, p, I.state_from_conditions(bad.n_tet, cond), drop_tol=0.1, max_steps=3)
    for _ in range(200):
        srv.step()
        if srv.status(rid).state == 4:
            break
        time.sleep(0.01)
    assert srv.status(rid).state == 4
    with pytest.raises(H.HGKSError):
        srv.collect(rid)


def test_server_compact_scheme_with_gradients_equals_alone(cuda):
    """The compact scheme carries G: served results (Q and G, caller order) equal the solve alone."""
    import torch
    kw = dict(scheme=1, krylov_dim=6, restarts=2, jacobi_sweeps=2)
    shared = H.hgks_default_params(**kw)
    srv = H.hgks_server(shared, hbm_budget_bytes=1 << 30, max_inflight=4)
    probs = []
    for k, (m, cond) in enumerate([(I.sphere_mesh(3, 4, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA),
                                    I.sphere_conditions(0.25, Re=118.0)),
                                   (I.cavity_mesh(3, seed=I.BASE_SEED + 23), I.cavity_conditions(0.2, 100.0))]):
        Q0, G0 = I.smooth_state(m, seed=I.BASE_SEED + 95 + k, amp=0.02,
                                base=(1.0, cond["u_inf"][0] + 0.03, 0.02, -0.01, cond["p_inf"]))
        p = H.hgks_default_params(**{**cond, "Pr": 0.72, **kw})
        rid = srv.submit(m, p, Q0, G0, drop_tol=0.3, max_steps=8)
        probs.append((m, p, Q0, G0, rid))
    while True:
        fin, run, wait = srv.step()
        if run == 0 and wait == 0:
            break
        if run == 0:
            time.sleep(0.005)
    for m, p, Q0, G0, rid in probs:
        st = srv.status(rid)
        Qs, Gs = srv.collect(rid, with_gradients=True)
        hm = H.hgks_mesh_create(m, scheme_mask=2)
        Qd, Gd = hm.to_internal(Q0), hm.to_internal(G0)
        info, _, _ = H.hgks_solve_steady(hm, p, Qd, Gd, drop_tol=0.3, max_steps=8)
        torch.cuda.synchronize()
        assert st.solve.steps == info.steps
        Qa, Ga = hm.to_caller(Qd), hm.to_caller(Gd)
        assert np.linalg.norm(Qs - Qa) <= 1e-9 * np.linalg.norm(Qa)
        assert np.linalg.norm(Gs - Ga) <= 1e-9 * np.linalg.norm(Ga)


def test_server_with_one_slot_runs_requests_in_order(cuda):
    """max_inflight = 1: one request at a time, admitted in arrival order."""
    probs = problems()[:3]
    srv = H.hgks_server(H.hgks_default_params(**KW), hbm_budget_bytes=1 << 30, max_inflight=1)
    ids = [srv.submit(m, p, Q0, drop_tol=DROP, max_steps=6) for _, m, _, p, Q0 in probs]
    while True:
        fin, run, wait = srv.step()
        assert run <= 1
        if run == 0 and wait == 0:
            break
        if run == 0:
            time.sleep(0.005)
    st = [srv.status(i) for i in ids]
    assert all(s.state == 3 for s in st)
    assert st[0].t_admit <= st[1].t_admit <= st[2].t_admit
    assert st[0].t_done <= st[1].t_admit and st[1].t_done <= st[2].t_admit


def _drain(srv):
    while True:
        fin, run, wait = srv.step()
        if run == 0 and wait == 0:
            return
        if run == 0:
            time.sleep(0.005)


def test_a_failing_request_leaves_the_others_bit_for_bit(cuda):
    """A request whose state holds a NaN fails (non-finite residual) while the
    requests beside it end exactly as they end without it: a mesh's arithmetic
    in the arena does not depend on its neighbours."""
    probs = problems()[:3]
    shared = H.hgks_default_params(**KW)

    def serve(with_bad):
        srv = H.hgks_server(shared, hbm_budget_bytes=1 << 30, max_inflight=8)
        ids = [srv.submit(m, p, Q0, drop_tol=DROP, max_steps=10) for _, m, _, p, Q0 in probs]
        bad = None
        if with_bad:
            _, m, _, p, Q0 = problems()[4]
            Qn = Q0.copy()
            Qn[7, 0] = np.nan
            bad = srv.submit(m, p, Qn, drop_tol=DROP, max_steps=10)
        _drain(srv)
        out = [srv.collect(i)[0] for i in ids]
        st = srv.status(bad) if with_bad else None
        return out, st

    ref, _ = serve(False)
    mixed, st_bad = serve(True)
    assert st_bad.state == 3 and st_bad.status == H.HGKS_ERR_NONPHYSICAL
    for a, b in zip(ref, mixed):
        assert np.array_equal(a, b)


def test_cancel_queued_and_running_requests(cuda):
    probs = problems()[:3]
    srv = H.hgks_server(H.hgks_default_params(**KW), hbm_budget_bytes=1 << 30, max_inflight=1)
    ids = [srv.submit(m, p, Q0, drop_tol=1e-12, max_steps=40) for _, m, _, p, Q0 in probs]
    for _ in range(2000):                   # until the first request runs
        srv.step()
        if srv.status(ids[0]).state == 2:
            break
        time.sleep(0.002)
    srv.step()
    srv.cancel(ids[0])                     # running: leaves with its state at the next round
    srv.cancel(ids[2])                     # waiting: dropped
    _drain(srv)
    s0, s1, s2 = (srv.status(i) for i in ids)
    assert s0.status == H.HGKS_ERR_CANCELLED and 0 < s0.solve.steps < 40
    assert s1.state == 3 and s1.status == H.HGKS_ERR_NOT_CONVERGED and s1.solve.steps == 40
    assert s2.status == H.HGKS_ERR_CANCELLED
    Q0c, _ = srv.collect(ids[0])           # the cancelled running request's state at cancellation
    assert np.isfinite(Q0c).all()
    with pytest.raises(H.HGKSError):
        srv.collect(ids[2])


def test_cancel_from_another_thread_while_rounds_run(cuda):
    """hgks_server_cancel may come from any thread while another drives the rounds:
    requests cancelled at arbitrary moments (waiting for their build, built, being
    admitted, running) all end, cancelled or finished, and the others end normally."""
    import threading
    probs = problems()
    srv = H.hgks_server(H.hgks_default_params(**KW), hbm_budget_bytes=1 << 30, max_inflight=1)
    ids = [srv.submit(m, p, Q0, drop_tol=DROP, max_steps=4) for _ in range(3) for _, m, _, p, Q0 in probs]
    victims = set(ids[1::2])

    def canceller():
        rng = np.random.default_rng(5)
        for rid in sorted(victims):
            time.sleep(float(rng.uniform(0.0, 0.01)))
            srv.cancel(rid)
    t = threading.Thread(target=canceller)
    t.start()
    while t.is_alive():
        fin, run, wait = srv.step()
        if run == 0:
            time.sleep(0.001)
    t.join()
    _drain(srv)
    for rid in ids:
        st = srv.status(rid)
        assert st.state == 3, (rid, st.state)
        if rid in victims:
            assert st.status in (H.HGKS_OK, H.HGKS_ERR_NOT_CONVERGED, H.HGKS_ERR_CANCELLED)
        else:
            assert st.status in (H.HGKS_OK, H.HGKS_ERR_NOT_CONVERGED), (rid, st.status)
    assert any(srv.status(r).status == H.HGKS_ERR_CANCELLED for r in victims)


def test_served_request_matches_the_oracle_solve(cuda):
    """A request served beside others (FP64 server) ends in the state the oracle's
    own steady solve (Algorithm 1, orc_solve_steady) reaches from the same start:
    the 3,456-tet inviscid sphere to a 1e-3 drop of the density residual, the
    same step count and the state within a relative L2 of 1e-9."""
    import oracle as O
    m = I.sphere_mesh(4, 6, stretch=1.3)
    cond = I.sphere_conditions(0.3)
    kw = dict(scheme=0, krylov_dim=10, restarts=3, jacobi_sweeps=2)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    drop, max_steps = 1e-3, 400
    om = O.OracleMesh(m)
    Qo, _, hist_o, conv_o = om.solve_steady(O.make_params(**cond, **kw), Q0, drop=drop, max_steps=max_steps)
    assert conv_o
    srv = H.hgks_server(H.hgks_default_params(**kw), hbm_budget_bytes=int(2e9), max_inflight=4)
    # two other requests run beside it
    others = [(I.cavity_mesh(3, seed=I.BASE_SEED + 31), I.cavity_conditions(0.2, 80.0)),
              (I.sphere_mesh(3, 6, stretch=1.25), I.sphere_conditions(0.45, aoa_deg=8.0))]
    for mo, co in others:
        srv.submit(mo, H.hgks_default_params(**{**co, "Pr": 0.72 if co["viscous"] else 1.0, **kw}),
                   I.state_from_conditions(mo.n_tet, co), drop_tol=drop, max_steps=50)
    rid = srv.submit(m, H.hgks_default_params(**cond, **kw), Q0, drop_tol=drop, max_steps=max_steps)
    t0 = time.time()
    while srv.status(rid).state < 3 and time.time() - t0 < 300:
        srv.step()
    st = srv.status(rid)
    assert st.status == 0 and st.solve.converged and st.solve.steps == len(hist_o) - 1, (st.solve.steps, len(hist_o) - 1)
    Q, _ = srv.collect(rid)
    assert np.linalg.norm(Q - Qo) <= 1e-9 * np.linalg.norm(Qo)
