"""The serving runtime: continuous batching of mixed residual/VJP requests
through the persistent kernel.

  * every request's result is identical alone and in the mix (bitwise);
  * FP64 residuals and VJPs equal the standalone kernels bitwise, FP32
    residuals meet the FP32 bars against the oracle;
  * Chandrashekar's flux in the same stream as Ranocha's, against the
    oracle's Chandrashekar flux;
  * admission under a budget that holds one request at a time, oversize
    rejection (SFH_ENOMEM), unknown tickets, a bounded drain timeout, a
    relaunch after the persistent kernel idled out, a per-request domain
    error that leaves the other requests intact.
"""
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from paper_2306_11665_gb300.serve import Server
from tests._helpers import fp32_check, rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _wait(srv, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serving timed out"
        time.sleep(0.0005)
    return out


def _make_requests(seed=0):
    """A mixed batch: degrees 2..8, both node sets, FP64/FP32/mixed residuals and VJPs."""
    rng = np.random.default_rng(seed)
    reqs = []
    specs = [(2, 0, "fp32k", 300), (3, 1, "fp64", 97), (4, 0, "fp32k", 500), (5, 0, "vjp", 64),
             (6, 1, "fp32mix", 40), (7, 1, "fp64", 33), (8, 0, "fp32k", 17), (4, 1, "vjp", 70),
             (3, 0, "fp64", 200), (2, 1, "vjp", 150)]
    for p, kind, prec, ne in specs:
        N = int(np.ceil(ne ** (1 / 3)))
        u, Ja = I.workload(3, p, kind, N, n_elem=ne, seed0=int(rng.integers(2, 1000)))
        lam = I.cotangent(u.shape, seed=int(rng.integers(1, 1000))) if prec == "vjp" else None
        reqs.append(dict(p=p, nodes=kind, prec=prec, u=u, Ja=Ja, lam=lam))
    return reqs


def _to_dev(r):
    dt = torch.float64 if r["prec"] in ("fp64", "vjp") else torch.float32
    u = torch.from_numpy(r["u"]).to(dt).cuda()
    Ja = torch.from_numpy(r["Ja"]).cuda()
    lam = torch.from_numpy(r["lam"]).cuda() if r["lam"] is not None else None
    return u, Ja, lam, torch.empty_like(u)


PREC = {"fp64": A.SFH_FP64, "fp32k": A.SFH_FP32_KAHAN, "fp32mix": A.SFH_FP32_MIXED, "vjp": A.SFH_FP64}


def _submit(srv, r, dev):
    u, Ja, lam, out = dev
    kind = A.SFH_REQ_VJP if r["prec"] == "vjp" else A.SFH_REQ_RESIDUAL
    return srv.submit(kind, r["p"], r["nodes"], PREC[r["prec"]], u, Ja, out, lam)


def test_alone_equals_in_the_mix_and_parity():
    reqs = _make_requests()
    devs = [_to_dev(r) for r in reqs]
    with Server(hbm_budget_bytes=8 << 30, max_inflight=16) as srv:
        # alone: one request at a time
        alone = []
        for r, dv in zip(reqs, devs):
            t = _submit(srv, r, dv)
            res = _wait(srv, [t])[t]
            assert res.status == A.SFH_OK
            alone.append(dv[3].clone())
        # in the mix: everything submitted at once, out of order
        for dv in devs:
            dv[3].fill_(float("nan"))
        order = list(range(len(reqs)))[::-1]
        tickets = [_submit(srv, reqs[i], devs[i]) for i in order]
        res = _wait(srv, tickets)
        assert all(x.status == A.SFH_OK for x in res.values())
        for i, dv in enumerate(devs):
            assert torch.equal(dv[3], alone[i]), i
    # against the standalone kernels and the oracle
    for r, dv, a in zip(reqs, devs, alone):
        p, kind = r["p"], r["nodes"]
        ctx = api.Context(3, p, kind, "euler")
        got = a.double().cpu().numpy()
        if r["prec"] == "vjp":
            assert torch.equal(a, ctx.vjp(dv[0], dv[1], dv[2]))
            ref = O.vjp_sf(3, p, kind, O.FLUX_EULER, r["u"], r["Ja"], r["lam"])
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        elif r["prec"] == "fp64":
            # the standalone FP64 path may pick another kernel (another
            # summation order) for a small mesh: equal to round-off
            sa = ctx.volume_residual(dv[0], dv[1], "fp64").double().cpu().numpy()
            assert rel_err_per_var(got, sa) <= 1e-13
            ref = O.volume_sf(3, p, kind, O.FLUX_EULER, r["u"], r["Ja"])
            assert rel_err_per_var(got, ref) <= 1e-12
        else:
            ref = O.volume_sf(3, p, kind, O.FLUX_EULER, r["u"], r["Ja"])
            u32 = I.to_fp32(r["u"]).astype(np.float64)
            ref_w = O.volume_sf(3, p, kind, O.FLUX_EULER, u32, r["Ja"])
            fp32_check(got, ref, ref_w, terms=O.volume_absterms(3, p, kind, O.FLUX_EULER, u32, r["Ja"]))


def test_chandrashekar_requests_in_a_mixed_stream():
    """Chandrashekar's flux through the server, interleaved with Ranocha
    requests of the same degrees and node sets: each result is the same alone
    and in the mix (bitwise); FP64 residuals and VJPs match the standalone
    kernels and the oracle's Chandrashekar flux at 1e-12, FP32 residuals meet
    the FP32 bars; a request naming Burgers' flux is refused."""
    rng = np.random.default_rng(11)
    specs = [(3, 0, "fp64", "ch", 90), (4, 1, "fp32k", "ch", 120), (5, 0, "vjp", "ch", 40),
             (4, 0, "fp32mix", "ch", 80), (4, 0, "fp64", "ra", 70), (6, 1, "fp32k", "ch", 30),
             (2, 1, "fp64", "ch", 150), (4, 1, "fp32k", "ra", 60)]
    reqs = []
    for p, kind, prec, fl, ne in specs:
        N = int(np.ceil(ne ** (1 / 3)))
        u, Ja = I.workload(3, p, kind, N, n_elem=ne, seed0=int(rng.integers(2, 1000)))
        lam = I.cotangent(u.shape, seed=int(rng.integers(1, 1000))) if prec == "vjp" else None
        reqs.append(dict(p=p, nodes=kind, prec=prec, u=u, Ja=Ja, lam=lam,
                         flux=A.SFH_FLUX_EULER_CHANDRASHEKAR if fl == "ch" else A.SFH_FLUX_EULER_RANOCHA))
    devs = [_to_dev(r) for r in reqs]

    def submit(srv, r, dv):
        u, Ja, lam, out = dv
        kind = A.SFH_REQ_VJP if r["prec"] == "vjp" else A.SFH_REQ_RESIDUAL
        return srv.submit(kind, r["p"], r["nodes"], PREC[r["prec"]], u, Ja, out, lam, flux=r["flux"])

    with Server(hbm_budget_bytes=8 << 30, max_inflight=16) as srv:
        alone = []
        for r, dv in zip(reqs, devs):
            t = submit(srv, r, dv)
            assert _wait(srv, [t])[t].status == A.SFH_OK
            alone.append(dv[3].clone())
        for dv in devs:
            dv[3].fill_(float("nan"))
        tickets = [submit(srv, reqs[i], devs[i]) for i in reversed(range(len(reqs)))]
        res = _wait(srv, tickets)
        assert all(x.status == A.SFH_OK for x in res.values())
        for i, dv in enumerate(devs):
            assert torch.equal(dv[3], alone[i]), i
        with pytest.raises(A.SfhError) as e:
            r = dict(reqs[0], flux=A.SFH_FLUX_BURGERS)
            submit(srv, r, devs[0])
        assert e.value.status == A.SFH_EINVAL
    for r, dv, a in zip(reqs, devs, alone):
        p, kind = r["p"], r["nodes"]
        ch = r["flux"] == A.SFH_FLUX_EULER_CHANDRASHEKAR
        of = O.FLUX_CHANDRASHEKAR if ch else O.FLUX_EULER
        ctx = api.Context(3, p, kind, "euler_chandrashekar" if ch else "euler")
        got = a.double().cpu().numpy()
        if r["prec"] == "vjp":
            assert torch.equal(a, ctx.vjp(dv[0], dv[1], dv[2]))
            ref = O.vjp_sf(3, p, kind, of, r["u"], r["Ja"], r["lam"])
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        elif r["prec"] == "fp64":
            sa = ctx.volume_residual(dv[0], dv[1], "fp64").double().cpu().numpy()
            assert rel_err_per_var(got, sa) <= 1e-13
            ref = O.volume_sf(3, p, kind, of, r["u"], r["Ja"])
            assert rel_err_per_var(got, ref) <= 1e-12
        else:
            ref = O.volume_sf(3, p, kind, of, r["u"], r["Ja"])
            u32 = I.to_fp32(r["u"]).astype(np.float64)
            ref_w = O.volume_sf(3, p, kind, of, u32, r["Ja"])
            fp32_check(got, ref, ref_w, terms=O.volume_absterms(3, p, kind, of, u32, r["Ja"]))


def test_admission_budget_oversize_and_tickets():
    reqs = _make_requests(seed=1)[:4]
    devs = [_to_dev(r) for r in reqs]
    sizes = []
    for r in reqs:
        nn = (r["p"] + 1) ** 3
        esz = 8 if r["prec"] in ("fp64", "vjp") else 4
        b = r["u"].shape[0] * nn * (2 * 5 * esz + 72) + (r["u"].shape[0] * nn * 40 if r["prec"] == "vjp" else 0)
        sizes.append(b)
    budget = max(sizes)   # room for one request at a time
    with Server(hbm_budget_bytes=budget, max_inflight=4) as srv:
        tickets = [_submit(srv, r, dv) for r, dv in zip(reqs, devs)]
        res = _wait(srv, tickets)
        assert all(x.status == A.SFH_OK for x in res.values())
        # FIFO under the budget: each was admitted only after the previous finished
        ordered = [res[t] for t in tickets]
        for a, b in zip(ordered, ordered[1:]):
            assert b.t_admit_ns >= a.t_done_ns - 5_000_000   # host clock granularity of the admission loop
        for x in ordered:
            assert x.t_submit_ns <= x.t_admit_ns <= x.t_done_ns
        # a request alone larger than the budget
        big = _to_dev(_make_requests(seed=2)[2])
        with pytest.raises(A.SfhError) as e:
            _submit(srv, dict(p=4, nodes=0, prec="fp32k", u=None, Ja=None, lam=None),
                    (big[0].repeat(8, 1, 1).contiguous(), big[1].repeat(8, 1, 1, 1).contiguous(), None,
                     torch.empty_like(big[0].repeat(8, 1, 1))))
        assert e.value.status == A.SFH_ENOMEM
        with pytest.raises(A.SfhError) as e:
            srv.poll(123456789)
        assert e.value.status == A.SFH_EINVAL


def test_idle_relaunch_drain_timeout_and_domain_error():
    reqs = _make_requests(seed=3)
    devs = [_to_dev(r) for r in reqs]
    with Server(hbm_budget_bytes=8 << 30, max_inflight=8) as srv:
        t = _submit(srv, reqs[0], devs[0])
        _wait(srv, [t])
        time.sleep(0.05)          # the persistent CTAs idle out after 2 ms
        t = _submit(srv, reqs[1], devs[1])
        assert _wait(srv, [t])[t].status == A.SFH_OK
        # a drain that cannot finish in 0 ms reports a timeout, then completes
        big = [_submit(srv, r, dv) for r, dv in zip(reqs, devs)]
        with pytest.raises(A.SfhError) as e:
            srv.drain(0)
        assert e.value.status == A.SFH_ETIMEOUT
        srv.drain(60000)
        _wait(srv, big)
        # one request with a negative density: its own status only
        bad = dict(reqs[1])
        ubad = bad["u"].copy()
        ubad[0, 0, 3] = -1.0
        bad["u"] = ubad
        dbad = _to_dev(bad)
        tb = _submit(srv, bad, dbad)
        tg = _submit(srv, reqs[3], devs[3])
        res = _wait(srv, [tb, tg])
        assert res[tb].status == A.SFH_EDOMAIN
        assert res[tg].status == A.SFH_OK


def test_serve_stats_count_tiles_per_class():
    reqs = _make_requests()
    devs = [_to_dev(r) for r in reqs]
    with Server(hbm_budget_bytes=8 << 30, max_inflight=16) as srv:
        s0 = A.sfh_serve_stats(srv.handle)
        tickets = [_submit(srv, r, dv) for r, dv in zip(reqs, devs)]
        res = _wait(srv, tickets)
        assert all(x.status == A.SFH_OK for x in res.values())
        s1 = A.sfh_serve_stats(srv.handle)
    used = {"fp64": 0, "fp32k": 0, "fp32mix": 0, "vjp": 0}
    for r in reqs:
        used[r["prec"]] += 1
    for k, n in used.items():
        dt = s1["tiles"][k] - s0["tiles"][k]
        assert (dt > 0) == (n > 0), (k, dt, n)
        if n:
            assert s1["busy_s"][k] > s0["busy_s"][k]
    assert s1["claim_s"] >= s0["claim_s"]
