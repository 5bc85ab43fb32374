"""Continuous-batching server: parity with the oracle and the single-lattice path,
bit-identical results alone and in a mix, memory-based admission, host-side fault
injection (allocation failure), cancellation and step limits."""
import os

import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from paper_2310_14746_gb300.serving import Server
from hlbm_testutil import make_lattice, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


def field(n, period, ratio, shape=None):
    return inputs.regular_sphere_field(shape or n, period=period, radius_ratio=ratio)


def test_server_fp32_matches_single_lattice_and_oracle(oracle):
    """A 32^3 request served with FP32 storage: its velocity equals the single-lattice
    FP32 path run for the same number of steps, and the FP64 oracle within 1e-5."""
    vp = field(32, 16, 0.3)
    srv = Server(1 << 30, hb.HLBM_F32, 100)
    srv.submit(vp, tau=0.6, F=(1e-5, 0, 0), tol=1e-30, max_steps=400, want_u=True)
    (r,) = srv.run_until_idle()
    srv.close()
    assert r["status"] == hb.HLBM_ERR_NOT_CONVERGED and r["steps"] == 400
    lat = make_lattice(19, (32, 32, 32), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, 0.6, (1e-5, 0, 0), (0, 0, 0), varpi=vp)
    lat.step(400)
    _, u = lat.moments()
    st = lat.reduce()
    lat.close()
    np.testing.assert_allclose(r["u"], u, rtol=0, atol=1e-6 * np.abs(u).max())
    assert abs(r["k_app"] - st["k_app"]) <= 1e-6 * abs(st["k_app"])
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.run(oracle.equilibrium_state(19, (32, 32, 32)), vp.astype(np.float64), 0.6, (1e-5, 0, 0),
                     (0, 0, 0), 400)
    _, ur = oracle.moments(ref, (1e-5, 0, 0), (0, 0, 0))
    assert rel_inf(r["u"], ur) < 1e-5


@pytest.mark.parametrize("storage", [hb.HLBM_F16DEV, hb.HLBM_BF16DEV, hb.HLBM_F32])
def test_same_result_alone_and_in_mix(storage):
    """Each request's result (steps, permeability, residual, velocity field) is bit-identical
    when it runs alone and when it shares the batch with requests of other sizes that
    arrive, run and retire around it. The 96^3 request runs on the single-lattice kernels in a
    branch of the round's graph of its own, beside the tile kernels of the small ones."""
    fa = field(32, 16, 0.35)
    fb = field(64, 32, 0.2)
    fc = field((48, 40, 24), 8, 0.3)
    fd = field(96, 32, 0.25)
    kw = dict(tau=0.6, F=(1e-5, 0, 0), tol=1e-7, max_steps=3000, want_u=True)
    alone = {}
    for name, f in (("a", fa), ("b", fb), ("c", fc), ("d", fd)):
        srv = Server(1 << 30, storage, 100)
        srv.submit(f, tag=ord(name), **kw)
        (r,) = srv.run_until_idle()
        srv.close()
        alone[ord(name)] = r
    srv = Server(1 << 30, storage, 100)
    srv.submit(fb, tag=ord("b"), **kw)
    srv.pump()
    srv.pump()
    srv.submit(fa, tag=ord("a"), **kw)
    srv.submit(fd, tag=ord("d"), **kw)
    srv.pump()
    srv.submit(fc, tag=ord("c"), **kw)
    mixed = {r["tag"]: r for r in srv.run_until_idle()}
    srv.close()
    assert set(mixed) == set(alone)
    for t, r in alone.items():
        m = mixed[t]
        assert (m["status"], m["steps"]) == (r["status"], r["steps"])
        assert m["k_app"] == r["k_app"] and m["max_du"] == r["max_du"] and m["mass"] == r["mass"]
        np.testing.assert_array_equal(m["u"], r["u"])


def test_memory_admission_and_fault_injection():
    """A budget that fits two 32^3 slots: never more than two run at once, injected
    allocation failures make admission back off, and every request still completes."""
    vp = field(32, 16, 0.3)
    per_slot = 2 * 19 * 32 ** 3 * 2 + 32 ** 3 * 16
    srv = Server(int(2.5 * per_slot), hb.HLBM_F16DEV, 50)
    ids = [srv.submit(vp, tau=0.6, F=(1e-5, 0, 0), tol=1e-30, max_steps=200) for _ in range(5)]
    srv.inject_alloc_failures(3)
    seen = []
    results = []
    while True:
        a, w = srv.pump()
        seen.append(a)
        results += srv.poll()
        if a == 0 and w == 0:
            break
    srv.close()
    assert max(seen) <= 2
    assert sorted(r["id"] for r in results) == sorted(ids)
    assert all(r["status"] == hb.HLBM_ERR_NOT_CONVERGED and r["steps"] == 200 for r in results)
    ks = {r["k_app"] for r in results}
    assert len(ks) == 1  # identical requests, identical results


def test_persistent_allocation_failure_fails_request():
    """With nothing running and every allocation failing, a request is retried for a few
    rounds and then returned with HLBM_ERR_OOM (no hang)."""
    vp = field(32, 16, 0.3)
    srv = Server(1 << 30, hb.HLBM_F16DEV, 100)
    rid = srv.submit(vp, tol=1e-30, max_steps=200)
    srv.inject_alloc_failures(1000)
    rounds = 0
    res = []
    while True:
        a, w = srv.pump()
        res += srv.poll()
        rounds += 1
        if a == 0 and w == 0:
            break
        assert rounds < 100
    srv.close()
    assert [(r["id"], r["status"]) for r in res] == [(rid, hb.HLBM_ERR_OOM)]


def test_cancel_and_invalid_requests():
    vp = field(32, 16, 0.3)
    srv = Server(1 << 30, hb.HLBM_F16DEV, 100)
    a = srv.submit(vp, tol=1e-30, max_steps=10 ** 6)
    b = srv.submit(vp, tol=1e-30, max_steps=10 ** 6)
    srv.cancel(b)  # still waiting: cancelled at once
    srv.pump()
    srv.cancel(a)  # live: retired at the next round
    res = srv.run_until_idle()
    res += srv.poll()
    st = {r["id"]: r["status"] for r in res}
    assert st == {a: hb.HLBM_ERR_CANCELLED, b: hb.HLBM_ERR_CANCELLED}
    bad = vp.copy()
    bad[0, 0, 0] = 2.0
    with pytest.raises(hb.HlbmError):
        srv.submit(bad)
    with pytest.raises(hb.HlbmError):
        srv.submit(vp, tau=0.5)
    with pytest.raises(hb.HlbmError):
        srv.submit(vp, tol=0.0)
    big = Server(1 << 20, hb.HLBM_F16DEV, 100)
    with pytest.raises(hb.HlbmError) as e:
        big.submit(vp)
    assert e.value.status == hb.HLBM_ERR_OOM
    big.close()
    srv.close()


def test_converges_to_steady_state():
    """A dense 32^3 pack reaches max|du| < 1e-6 per 100 steps; the permeability it returns
    matches the single-lattice FP32 run to the same step count within FP16 error."""
    vp = field(32, 16, 0.45)
    srv = Server(1 << 30, hb.HLBM_F16DEV, 100)
    srv.submit(vp, tau=0.6, F=(1e-6, 0, 0), tol=1e-6, max_steps=200000)
    (r,) = srv.run_until_idle()
    srv.close()
    assert r["status"] == hb.HLBM_OK
    assert r["max_du"] < 1e-6
    lat = make_lattice(19, (32, 32, 32), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, 0.6, (1e-6, 0, 0), (0, 0, 0), varpi=vp)
    lat.step(r["steps"])
    st = lat.reduce()
    lat.close()
    assert abs(r["k_app"] - st["k_app"]) / st["k_app"] < 1e-2


def test_precision_ladder_reaches_tolerance():
    """A fast flow (period 64, r = 0.3 P: max|u| ~ 1e-2) cannot reach max|du| < 1e-6 in FP16
    storage (its rounding floor is ~6e-4 max|u|). With refinement the slot moves to FP32 at
    the floor and converges; its permeability agrees with an FP32-only server within 1 %."""
    vp = field(64, 64, 0.3)
    kw = dict(tau=0.6, F=(1e-6, 0, 0), tol=1e-6, max_steps=200000)
    srv = Server(4 << 30, hb.HLBM_F16DEV, 100)
    srv.submit(vp, **kw)
    (r,) = srv.run_until_idle()
    srv.close()
    assert r["status"] == hb.HLBM_OK, r
    assert r["final_storage"] == hb.HLBM_F32 and 0 < r["steps_low"] < r["steps"]
    ref_srv = Server(4 << 30, hb.HLBM_F32, 100)
    ref_srv.submit(vp, **kw)
    (ref,) = ref_srv.run_until_idle()
    ref_srv.close()
    assert ref["status"] == hb.HLBM_OK and ref["steps_low"] == 0
    assert abs(r["k_app"] - ref["k_app"]) / ref["k_app"] < 1e-2
    # without refinement the FP16 slot stalls above the tolerance
    off = Server(4 << 30, hb.HLBM_F16DEV, 100, refine=False)
    off.submit(vp, tau=0.6, F=(1e-6, 0, 0), tol=1e-6, max_steps=20000)
    (o,) = off.run_until_idle()
    off.close()
    assert o["status"] == hb.HLBM_ERR_NOT_CONVERGED and o["final_storage"] == hb.HLBM_F16DEV


@pytest.mark.parametrize("storage", [hb.HLBM_F16DEV, hb.HLBM_BF16DEV, hb.HLBM_F32])
@pytest.mark.parametrize("F", [(1e-5, 0.0, 0.0), (1e-5, 2e-6, -3e-6)])
@pytest.mark.parametrize("dims", [(32, 32, 32), (96, 40, 24), (50, 30, 20)])
def test_batched_slot_bit_identical_to_single_lattice(dims, F, storage):
    """A slot served without refinement holds, after 400 steps, the same velocity field bit for
    bit as the single-lattice path in the same storage: the batched kernels (paired 16-bit
    kernel with either load scheme, per-cell kernel) and the single-lattice kernels compute
    the same collision. nx = 50 gives 25 pairs per row, a tile with idle lanes."""
    nx, ny, nz = dims
    vp = inputs.regular_sphere_field((nx, ny, nz), period=10 if nx == 50 else 8, radius_ratio=0.3)
    srv = Server(1 << 30, storage, 100, refine=False)
    srv.submit(vp, tau=0.6, F=F, tol=1e-30, max_steps=400, want_u=True)
    (r,) = srv.run_until_idle()
    srv.close()
    assert r["status"] == hb.HLBM_ERR_NOT_CONVERGED and r["steps"] == 400
    lat = make_lattice(19, (nz, ny, nx), storage, hb.HLBM_TWO_LATTICE, 0.6, F, (0, 0, 0), varpi=vp)
    lat.step(400)
    _, u = lat.moments()
    lat.close()
    np.testing.assert_array_equal(r["u"], u)


@pytest.mark.parametrize("backfill,rounds", [(1e9, [4, 4, 4]), (1.0, [4, 4, 8]), (0.0, [4, 8, 12])])
def test_age_priority_changes_when_not_what(backfill, rounds):
    """Three equal 160^3 requests (4.1M cells each, above the 4M cells a round is always
    filled to) submitted in order, 400 steps each. A round runs the oldest request plus
    younger ones within (1 + backfill) times its cells: everything at once for a huge
    backfill, two at a time for 1, strictly one after another for 0. The results are
    bit-identical in every schedule."""
    vp = field(160, 32, 0.3)
    srv = Server(4 << 30, hb.HLBM_F16DEV, 100, backfill=backfill)
    ids = [srv.submit(vp, tol=1e-30, max_steps=400, want_u=True) for _ in range(3)]
    finished_round = {}
    n = 0
    results = []
    while True:
        a, w = srv.pump()
        n += 1
        for r in srv.poll():
            finished_round[r["id"]] = n
            results.append(r)
        if a == 0 and w == 0:
            break
    srv.close()
    assert all(r["steps"] == 400 for r in results)
    assert [finished_round[i] for i in ids] == rounds
    u0 = results[0]["u"]
    for r in results[1:]:
        np.testing.assert_array_equal(r["u"], u0)
        assert r["k_app"] == results[0]["k_app"]
