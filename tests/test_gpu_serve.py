"""Continuous-batching server: results must not depend on the batch they run in.

A request's result is a deterministic function of its controller's state (nominal, counter), its
state estimate and its (K, M, T): alone or in a mix of other controllers' requests, with or without
CUDA graphs, it must come out bit for bit the same, and equal to bssmppi_solve + bssmppi_shift on
a single handle within the update tolerance (rel 1e-4 / abs 1e-5; the two update kernels add the
weighted perturbations in different orders), with the minimum trajectory cost within the cost
tolerance (the two evaluate the tyre curve differently where fewer than four particles share a lane).
Served requests are also compared with the FP64 oracle sample by sample (costs, weights and
perturbations read back through bssmppi_server_capture).
"""
import time

import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402

T_MAX = 60


def _problem(i):
    kappa, length = workload.make_track(1000 + i, n_theta=1 << 13)
    p = workload.racing_problem(256, 16, 20, track_seed=0, noise_scale=2.0, seed=i)
    p.kappa, p.track_len = kappa, length
    return p


def _server(n_ctrl, **kw):
    s = bssmppi.server_create(n_ctrl, T_max=T_MAX, **kw)
    probs = [_problem(i) for i in range(n_ctrl)]
    for p in probs:
        bssmppi.server_add_controller(s, bssmppi.make_params(p))
    return s, probs


def _v0(i):
    v = np.zeros((T_MAX, 2), np.float32)
    v[:, 0] = 0.04 + 0.002 * i
    v[:, 1] = 0.1 * np.sin(np.arange(T_MAX) * 0.2 + i)
    return v


MIX = [(512, 8, 20), (2048, 32, 40), (4096, 64, 40), (1024, 128, 60), (700, 64, 20), (333, 8, 60),
       (4096, 32, 60), (8192, 64, 40), (1500, 128, 20), (64, 8, 40)]


def _x0(i):
    return np.array([9.0 + 0.1 * i, 0.05, 0.01, 0.02 * ((i % 5) - 2), 0.3 * ((i % 7) - 3), 3.0 * i], np.float32)


def _run(s, requests, ctr0=5):
    """requests: list of (ctrl, K, M, T). Resets the controllers, submits all, drains, returns
    {ctrl: (u0, v_after, counter_after, beta)}."""
    for c, *_ in requests:
        bssmppi.server_set_state(s, c, _v0(c), ctr0)
    for j, (c, K, M, T) in enumerate(requests):
        bssmppi.server_submit(s, c, _x0(c), K, M, T, req_id=1000 * c + j)
    bssmppi.server_drain(s, 60000)
    res = {r.ctrl_id: r for r in bssmppi.server_poll(s)}
    out = {}
    for c, *_ in requests:
        assert res[c].status == 0
        v, ctr = bssmppi.server_get_state(s, c, T_MAX)
        out[c] = (np.array(res[c].u0), v, ctr, res[c].beta)
    return out


def test_result_alone_equals_in_mix_and_without_graphs():
    s, _ = _server(len(MIX))
    try:
        mix = [(c, K, M, T) for c, (K, M, T) in enumerate(MIX)]
        together = _run(s, mix)
        for c, K, M, T in mix[:4] + mix[-2:]:
            alone = _run(s, [(c, K, M, T)])
            assert np.array_equal(alone[c][0], together[c][0]), c
            assert np.array_equal(alone[c][1], together[c][1]), c
            assert alone[c][2] == together[c][2] == 6
        st = bssmppi.server_get_stats(s)
        assert st["superseded"] == 0 and st["completed"] == st["submitted"]
    finally:
        bssmppi.server_destroy(s)
    s2, _ = _server(len(MIX), use_graphs=False, slots=1)
    try:
        eager = _run(s2, [(c, K, M, T) for c, (K, M, T) in enumerate(MIX)])
        for c in eager:
            assert np.array_equal(eager[c][0], together[c][0]) and np.array_equal(eager[c][1], together[c][1])
    finally:
        bssmppi.server_destroy(s2)
    s4, _ = _server(len(MIX), slots=4, max_batch=2)  # four batches in flight, two requests each
    try:
        four = _run(s4, [(c, K, M, T) for c, (K, M, T) in enumerate(MIX)])
        for c in four:
            assert np.array_equal(four[c][0], together[c][0]) and np.array_equal(four[c][1], together[c][1])
        assert bssmppi.server_get_stats(s4)["batches"] >= len(MIX) // 2
    finally:
        bssmppi.server_destroy(s4)


@pytest.mark.parametrize("K,M,T", [(4096, 64, 40), (512, 8, 20), (1024, 128, 60), (700, 33, 20)])
def test_server_matches_single_solve(K, M, T):
    s, probs = _server(3)
    try:
        got = _run(s, [(2, K, M, T)])[2]
    finally:
        bssmppi.server_destroy(s)
    p = probs[2]
    p.K, p.M, p.T = K, M, T
    c = bssmppi.Controller(p)
    bssmppi.set_counter(c.h, 5)
    v = torch.as_tensor(_v0(2)[:T], device="cuda").contiguous()
    u0 = torch.zeros(2, device="cuda")
    bssmppi.solve(c.h, torch.as_tensor(_x0(2), device="cuda"), None, v, u0)
    bssmppi.shift(c.h, v, 1)
    torch.cuda.synchronize()
    ctr = bssmppi.get_counter(c.h)
    S = c.buffer(bssmppi.BUF_S).cpu().numpy()
    c.close()
    ref_u0, ref_v = u0.cpu().numpy(), v.cpu().numpy()
    # The rollouts are the same arithmetic except the tyre curve: the single-solve kernel takes it
    # from its polynomial where one or two particles share a lane, the server from the library's
    # arctangent and sine (both within 4e-7 of sin(C atan x)). So the minimum trajectory cost agrees
    # within the cost tolerance of the parity tests, and bit for bit where four particles share a lane.
    if M > 64:
        assert np.float32(got[3]) == S.min()
    assert abs(float(got[3]) - float(S.min())) <= 1e-4 * max(1.0, abs(float(S.min())))
    assert np.all(np.abs(got[0] - ref_u0) <= 1e-5 + 1e-4 * np.abs(ref_u0))
    assert np.all(np.abs(got[1][:T] - ref_v) <= 1e-5 + 1e-4 * np.abs(ref_v))
    assert got[2] == ctr == 6


def test_two_constants_classes_batch_apart_and_match_their_single_solves():
    """Controllers whose vehicles or costs differ (here the mass, and for one controller cost weights
    on every state, whose class takes the kernel path that merges every mean) are batched by
    constants class: each batch's rollout kernels take that class's constants as a parameter, and
    the graph's kernel parameters are switched when a slot's class changes. Every request must still
    give, bit for bit, what it gives alone, with and without graphs, and match bssmppi_solve +
    bssmppi_shift."""
    n = 6
    s = bssmppi.server_create(n, T_max=T_MAX)
    probs = [_problem(i) for i in range(n)]
    for i, p in enumerate(probs):
        if i % 2:
            p.mass = 1200.0  # a lighter vehicle: a second constants class
        if i == 5:
            p.Q = p.Qf = (1.0, 0.5, 0.2, 1.0, 0.1, 1e-4)  # every state weighted: a third class
        bssmppi.server_add_controller(s, bssmppi.make_params(p))
    reqs = [(c, 1024 + 256 * c, (8, 32, 64, 128, 64, 32)[c], (20, 40, 60, 20, 40, 60)[c]) for c in range(n)]
    try:
        together = _run(s, reqs)
        for _ in range(2):  # the classes alternate between batches: the graph's parameters follow
            again = _run(s, reqs)
            for c in together:
                assert np.array_equal(again[c][0], together[c][0]) and np.array_equal(again[c][1], together[c][1])
        for r in reqs[:3]:
            alone = _run(s, [r])
            assert np.array_equal(alone[r[0]][0], together[r[0]][0])
            assert np.array_equal(alone[r[0]][1], together[r[0]][1])
        assert bssmppi.server_get_stats(s)["batches"] >= 2 * 3 + 3
    finally:
        bssmppi.server_destroy(s)
    s2 = bssmppi.server_create(n, T_max=T_MAX, use_graphs=False, slots=1)
    try:
        for p in probs:
            bssmppi.server_add_controller(s2, bssmppi.make_params(p))
        eager = _run(s2, reqs)
    finally:
        bssmppi.server_destroy(s2)
    for c, K, M, T in reqs:
        assert np.array_equal(eager[c][0], together[c][0]) and np.array_equal(eager[c][1], together[c][1])
        p = probs[c]
        p.K, p.M, p.T = K, M, T
        h = bssmppi.Controller(p)
        try:
            bssmppi.set_counter(h.h, 5)
            v = torch.as_tensor(_v0(c)[:T], device="cuda").contiguous()
            u0 = torch.zeros(2, device="cuda")
            bssmppi.solve(h.h, torch.as_tensor(_x0(c), device="cuda"), None, v, u0)
            bssmppi.shift(h.h, v, 1)
            torch.cuda.synchronize()
            S = h.buffer(bssmppi.BUF_S).cpu().numpy()
        finally:
            h.close()
        assert abs(float(together[c][3]) - float(S.min())) <= 1e-4 * max(1.0, abs(float(S.min()))), c
        ref_v = v.cpu().numpy()
        assert np.all(np.abs(together[c][1][:T] - ref_v) <= 1e-5 + 1e-4 * np.abs(ref_v)), c


ORACLE_MIX = [(4096, 64, 40), (1024, 128, 60), (700, 33, 20), (512, 8, 20), (2048, 32, 60)]


def test_served_requests_match_the_oracle():
    """Each request of a mixed batch against the FP64 oracle's solve of the same controller state and
    counter followed by its one-step shift (Alg. 1, "ExecuteCommand" and the warm start): every
    sample's perturbation (atol 1e-6) and cost (rel 1e-4, away from the collision indicator's jump),
    the weights against the oracle's weights of the served costs (rel 1e-5 / abs 1e-7), the minimum
    cost, u0 and the shifted nominal against the oracle's own (rel 1e-4 / abs 1e-5 plus twice the
    first-order bound that the measured cost differences imply, as in the single-solve parity)."""
    s, probs = _server(len(ORACLE_MIX))
    ctr0 = 11
    try:
        caps = {}
        for c, (K, M, T) in enumerate(ORACLE_MIX):
            bssmppi.server_set_state(s, c, _v0(c), ctr0)
            caps[c] = bssmppi.server_capture(s, c, K, T)
        for c, (K, M, T) in enumerate(ORACLE_MIX):
            bssmppi.server_submit(s, c, _x0(c), K, M, T, req_id=c)
        bssmppi.server_drain(s, 60000)
        res = {r.ctrl_id: r for r in bssmppi.server_poll(s)}
        after = {c: bssmppi.server_get_state(s, c, T_MAX) for c in range(len(ORACLE_MIX))}
        assert bssmppi.server_get_stats(s)["max_batch_seen"] >= 2  # they did share a batch
    finally:
        bssmppi.server_destroy(s)
    for c, (K, M, T) in enumerate(ORACLE_MIX):
        r = res[c]
        assert r.status == 0 and (r.K, r.M, r.T) == (K, M, T)
        S, w, eps = (a.astype(np.float64) for a in caps[c].result(K, T))
        p = probs[c]
        p.K, p.M, p.T = K, M, T
        v = _v0(c)[:T]
        ref = oracle.Oracle(p).solve(_x0(c), v, ctr0, threads=oracle.host_threads())
        assert np.all(np.abs(eps - ref["eps"]) <= 1e-6), c
        ok = ref["margin"] > 1e-4
        assert (~ok).sum() <= max(2, K // 100)
        scale = np.maximum(np.abs(ref["S"]), 1.0)
        dS = S - ref["S"]
        assert np.all(np.abs(dS[ok]) <= 1e-4 * scale[ok]), (c, np.max(np.abs(dS[ok]) / scale[ok]))
        lam = float(np.float32(p.lam))
        w_iso, _, _ = oracle.optimal_control(S, v.astype(np.float64)[None] + eps, lam)
        assert np.all(np.abs(w - w_iso) <= 1e-7 + 1e-5 * w_iso), c
        beta_ref = ref["diag"][0]
        assert abs(r.beta - beta_ref) <= 1e-4 * max(1.0, abs(beta_ref)), c
        dSc = np.where(ok, dS, 0.0)
        dev = np.abs(dSc - np.sum(ref["w"] * dSc)) / lam
        bound = np.einsum("k,kti->ti", ref["w"] * dev, np.abs(ref["u"] - ref["v_plus"][None]))
        vp = ref["v_plus"]
        tol = 1e-5 + 1e-4 * np.abs(vp) + 2 * bound
        assert np.all(np.abs(np.array(r.u0) - vp[0]) <= tol[0]), c
        shifted, tol_s = vp.copy(), tol.copy()
        shifted[:-1], tol_s[:-1] = vp[1:], tol[1:]
        v_after, ctr_after = after[c]
        err = np.abs(v_after[:T] - shifted)
        assert np.all(err <= tol_s), (c, err.max())
        assert np.array_equal(v_after[T:], _v0(c)[T:])  # entries past the request's horizon untouched
        assert ctr_after == ctr0 + 1
        print(f"[serve vs oracle] K={K} M={M} T={T}: S max rel {np.max(np.abs(dS[ok]) / scale[ok]):.2e}, "
              f"beta {r.beta:.6g} vs {beta_ref:.6g}, shifted v+ max err {err.max():.2e} (bound {bound.max():.2e}), "
              f"indicator-margin exclusions {(~ok).sum()}")


def test_capture_that_does_not_fit_copies_nothing():
    """A capture buffer smaller than K (2 + 2T) floats reports -1 and is left untouched; the request
    itself completes normally, and a later capture of the controller works."""
    s, _ = _server(1)
    try:
        bssmppi.server_set_state(s, 0, _v0(0), 3)
        small = bssmppi.server_capture(s, 0, 64, 20)  # room for K = 64, T = 20
        small.buf[:] = 7.0
        bssmppi.server_submit(s, 0, _x0(0), 512, 16, 20, req_id=1)
        bssmppi.server_drain(s, 60000)
        res = bssmppi.server_poll(s)
        assert [r.status for r in res] == [0]
        assert small.written.value == -1 and np.all(small.buf == 7.0)
        with pytest.raises(bssmppi.BssmppiError):
            small.result(512, 20)
        ok = bssmppi.server_capture(s, 0, 512, 20)
        bssmppi.server_submit(s, 0, _x0(0), 512, 16, 20, req_id=2)
        bssmppi.server_drain(s, 60000)
        bssmppi.server_poll(s)
        S, w, eps = ok.result(512, 20)
        assert abs(float(w.sum()) - 1.0) < 1e-5 and np.all(np.isfinite(S)) and eps.shape == (512, 20, 2)
    finally:
        bssmppi.server_destroy(s)


def test_newer_request_replaces_pending_one_and_every_request_gets_a_result():
    s, _ = _server(2, max_batch=1, slots=1)
    try:
        for c in range(2):
            bssmppi.server_set_state(s, c, _v0(c), 0)
        ids = []
        for j in range(6):  # a burst for controller 0: the first runs, later ones replace each other
            bssmppi.server_submit(s, 0, _x0(0), 8192, 128, 60, req_id=j)
            ids.append(j)
        bssmppi.server_submit(s, 1, _x0(1), 256, 16, 20, req_id=99)
        bssmppi.server_drain(s, 60000)
        res = bssmppi.server_poll(s)
        got = sorted(r.req_id for r in res)
        assert got == sorted(ids + [99])
        ok = [r for r in res if r.status == 0]
        replaced = [r for r in res if r.status != 0]
        assert len(ok) >= 2 and len(replaced) >= 1
        assert all(r.status == -5 for r in replaced)  # BSSMPPI_EBUSY
        assert max(r.req_id for r in ok if r.ctrl_id == 0) == 5  # the newest always runs
        _, ctr0 = bssmppi.server_get_state(s, 0, T_MAX)
        assert ctr0 == len([r for r in ok if r.ctrl_id == 0])
        for r in ok:
            assert r.t_submit_us <= r.t_start_us <= r.t_done_us
    finally:
        bssmppi.server_destroy(s)


def test_admission_respects_hbm_budget():
    # 4 MiB per slot holds 3 requests of K=4096, T=40 (1.31 MB of perturbations + costs each)
    s, _ = _server(12, hbm_budget_bytes=8 << 20)
    try:
        for c in range(12):
            bssmppi.server_set_state(s, c, _v0(c), 0)
        for c in range(12):
            bssmppi.server_submit(s, c, _x0(c), 4096, 64, 40, req_id=c)
        bssmppi.server_drain(s, 60000)
        res = bssmppi.server_poll(s)
        assert sorted(r.req_id for r in res if r.status == 0) == list(range(12))
        st = bssmppi.server_get_stats(s)
        assert 1 <= st["max_batch_seen"] <= 3 and st["batches"] >= 4
    finally:
        bssmppi.server_destroy(s)


def test_server_rejects_bad_slot_counts():
    for slots in (0, 9):
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.server_create(2, T_max=T_MAX, slots=slots)


def test_server_rejects_bad_requests():
    s, _ = _server(1, hbm_budget_bytes=2 << 20)
    try:
        x0 = _x0(0)
        for args in ((0, x0, 256, 256, 20), (0, x0, 256, 16, 61), (3, x0, 256, 16, 20), (0, x0, 0, 16, 20),
                     (0, x0, 1 << 17, 64, 60)):
            with pytest.raises(bssmppi.BssmppiError):
                bssmppi.server_submit(s, *args, req_id=1)
    finally:
        bssmppi.server_destroy(s)
