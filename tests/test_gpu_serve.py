"""Serving loop: results equal solo runs bit for bit, alone and in a mix;
admission by memory; back-pressure, fault injection and timeouts (all
failures are made on the host: no GPU fault is involved)."""
import time

import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu


def _requests(orc, spec, seed=0):
    sizes = [37, 300, 96, 711, 64, 150]
    out = []
    for i, n in enumerate(sizes):
        truth, obs = make_obs(orc, spec, n, seed=100 + i + seed)
        sig = 1e-3 * (truth[:, 7] + truth[:, 8])
        w = np.repeat((1 / sig)[:, None], 4, 1)
        out.append(dict(obs=obs.astype(np.float32), npop=64 if i % 2 else 128, ngen=10 + 5 * i,
                        pid0=10_000 * i, polish=3 if i % 3 == 0 else 0, w=w))
    return out


def _solo(gpu, pb, r):
    ob = torch.tensor(r["obs"], device="cuda")
    ga = gpu.GaSettings(npop=r["npop"], ngen=r["ngen"], seed=5)
    best, chi2 = gpu.ga_invert_batch(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, pixel_id0=r["pid0"])
    if r["polish"]:
        best, chi2 = gpu.lm_polish(pb, ob, best, gi.PRIOR_LO, gi.PRIOR_HI, iters=r["polish"],
                                   w=torch.tensor(r["w"], device="cuda"))
    torch.cuda.synchronize()
    return best.cpu().numpy(), chi2.cpu().numpy()


def _submit(gpu, srv, r):
    return srv.submit(r["obs"], gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=r["npop"], ngen=r["ngen"], seed=5),
                      pixel_id0=r["pid0"], polish_iters=r["polish"], polish_w=r["w"] if r["polish"] else None)


def test_results_equal_solo_runs_alone_and_mixed(gpu, orc):
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    reqs = _requests(orc, spec)
    solo = [_solo(gpu, pb, r) for r in reqs]
    # all at once: they are admitted together and overlap on the device
    with gpu.Server(pb, arena_bytes=64 << 20, max_inflight=4, small_pixels=100) as srv:
        tickets = [_submit(gpu, srv, r) for r in reqs]
        got = [srv.poll(t) for t in tickets]
    for (b, c), g in zip(solo, got):
        assert np.array_equal(b, g["best"]) and np.array_equal(c, g["chi2"])
        assert g["latency_ns"] >= g["queue_ns"] >= 0
    # one at a time on a single slot
    with gpu.Server(pb, arena_bytes=64 << 20, max_inflight=1) as srv:
        for r, (b, c) in zip(reqs, solo):
            g = srv.poll(_submit(gpu, srv, r))
            assert np.array_equal(b, g["best"]) and np.array_equal(c, g["chi2"])


def test_admission_by_memory(gpu, orc):
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    reqs = []
    for i in range(4):
        truth, obs = make_obs(orc, spec, 400, seed=300 + i)
        reqs.append(dict(obs=obs.astype(np.float32), npop=64, ngen=30, pid0=1000 * i, polish=0, w=None))
    per_req = 400 * (4 * 128 * 4 + 9 * 8 + 8) + 3 * 256
    # the arena holds 1.5 requests: admission must wait for memory, one at a time
    with gpu.Server(pb, arena_bytes=int(1.5 * per_req), max_inflight=4) as srv:
        tickets = [_submit(gpu, srv, r) for r in reqs]
        peak = 0
        t0 = time.time()
        while time.time() - t0 < 60:
            st = srv.stats()
            peak = max(peak, st["running"])
            assert st["arena_used"] <= st["arena_bytes"]
            if st["queued"] == 0 and st["running"] == 0:
                break
            time.sleep(0.001)
        res = [srv.poll(t) for t in tickets]
    assert peak == 1
    assert all(r["status"] == 0 for r in res)
    # later requests waited in the queue for the earlier ones' memory
    assert res[-1]["queue_ns"] > res[0]["queue_ns"]


def test_backpressure_fault_injection_and_timeouts(gpu, orc):
    from paper_1208_0302_gb300 import _lib
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    reqs = _requests(orc, spec, seed=2)
    with gpu.Server(pb, arena_bytes=64 << 20, max_inflight=2, max_queue=64,
                    fail_next_admissions=1) as srv:
        t_fail = _submit(gpu, srv, reqs[0])
        t_ok = _submit(gpu, srv, reqs[1])
        with pytest.raises(_lib.GenesisError) as e:
            srv.poll(t_fail)
        assert e.value.code == _lib.ME_ENOMEM
        assert srv.poll(t_ok)["status"] == 0
        with pytest.raises(_lib.GenesisError) as e:
            srv.poll(123456)
        assert e.value.code == _lib.ME_ENOTFOUND
        big = dict(reqs[3], ngen=400)
        t_big = _submit(gpu, srv, big)
        with pytest.raises(_lib.GenesisError) as e:
            srv.poll(t_big, timeout_ms=1)
        assert e.value.code == _lib.ME_ETIMEOUT
        with pytest.raises(_lib.GenesisError) as e:
            srv.poll(t_big, timeout_ms=0)
        assert e.value.code == _lib.ME_EPENDING
        assert srv.poll(t_big, timeout_ms=-1)["status"] == 0
    # request larger than the arena, and a full queue
    with gpu.Server(pb, arena_bytes=1 << 20, max_inflight=1, max_queue=2) as srv:
        with pytest.raises(_lib.GenesisError) as e:
            _submit(gpu, srv, reqs[3])
        assert e.value.code == _lib.ME_EINVAL
        codes = []
        tickets = []
        for _ in range(8):
            try:
                tickets.append(_submit(gpu, srv, dict(reqs[2], ngen=200)))
            except _lib.GenesisError as err:
                codes.append(err.code)
        assert _lib.ME_EAGAIN in codes
        for t in tickets:
            srv.poll(t)
    # destroy with queued work does not hang
    srv = gpu.Server(pb, arena_bytes=64 << 20, max_inflight=1)
    for r in reqs:
        _submit(gpu, srv, r)
    srv.close()


def test_invalid_requests_rejected(gpu, orc):
    from paper_1208_0302_gb300 import _lib
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    obs = np.zeros((10, 4, 128), np.float32)
    with gpu.Server(pb, arena_bytes=1 << 22) as srv:
        with pytest.raises(_lib.GenesisError):
            srv.submit(obs, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=40, ngen=2))
        lo = gi.PRIOR_LO.copy()
        lo[5] = -1.0
        with pytest.raises(_lib.GenesisError):
            srv.submit(obs, lo, gi.PRIOR_HI, gpu.GaSettings(npop=32, ngen=2))
    with pytest.raises(_lib.GenesisError):
        gpu.Server(pb, arena_bytes=100)
