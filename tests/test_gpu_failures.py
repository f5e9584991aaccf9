"""Failure detection without a GPU fault, request cancellation and GA
checkpoint / resume, through the C ABI."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_1704_06258_gb300 import binding, synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance, Server, UsaphmpError

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_bounded_waits_give_up_and_the_context_survives():
    rc, status, elapsed = binding.selftest_wait_timeout(20_000_000)      # 20 ms
    # ETIMEOUT: the timeout bit is set in the status word and no wait succeeded
    assert binding.ERRORS.get(rc) == "ETIMEOUT"
    assert status != 0 and not status & 0x80000000
    assert 20_000_000 <= elapsed < 2_000_000_000
    inst = synth.urand200(seed=3, n=50, p=4)
    hubs, S = synth.random_population(4, inst.n, inst.p, 5)
    with Instance.from_instance(inst) as gi:                              # the GPU still works
        assert np.isfinite(gi.eval(hubs, S)).all()


def test_injected_allocation_failures_report_enomem():
    inst = synth.urand200(seed=5, n=80, p=6)
    hubs, S = synth.random_population(6, inst.n, inst.p, 7)
    failures = 0
    try:
        for after in range(0, 40, 3):
            binding.debug_fail_allocations(after)
            try:
                with Instance.from_instance(inst) as gi:
                    gi.eval(hubs, S)
                    gi.solve(2, 1)
            except UsaphmpError as e:
                assert e.name == "ENOMEM", str(e)
                failures += 1
    finally:
        binding.debug_fail_allocations(-1)
    assert failures >= 3
    with Instance.from_instance(inst) as gi:
        assert np.isfinite(gi.eval(hubs, S)).all()


def _drain(server, tickets):
    res = {}
    for _ in range(10000):
        server.step()
        for t in list(tickets):
            try:
                r = server.poll(t)
            except UsaphmpError as e:
                res[t] = e.name
                tickets.remove(t)
                continue
            if r is not None:
                res[t] = r
                tickets.remove(t)
        if not tickets:
            return res
    raise AssertionError("server did not finish")


def test_cancelled_requests_free_their_slots_and_leave_the_others_alone():
    reqs = [synth.clustered(seed=7400 + r, n=n, p=p) for r, (n, p) in enumerate([(120, 5), (200, 8), (90, 4)])]
    with Server(4 * GB, max_active=2, path=PATH_SPLIT_BF16) as s:
        alone = []
        for k, inst in enumerate(reqs):
            t = s.submit(inst.W, inst.C, inst.p, islands=2, island_size=16, generations=40, seed=10 + k)
            alone.append(_drain(s, [t])[t])
    with Server(4 * GB, max_active=2, path=PATH_SPLIT_BF16) as s:
        tickets = [s.submit(i.W, i.C, i.p, islands=2, island_size=16, generations=40, seed=10 + k)
                   for k, i in enumerate(reqs)]
        active, pending = s.step()
        assert (active, pending) == (2, 1)
        s.cancel(tickets[0])                 # running
        s.cancel(tickets[2])                 # still queued
        with pytest.raises(UsaphmpError):
            s.cancel(tickets[2])             # already cancelled
        with pytest.raises(UsaphmpError):
            s.cancel(987654)                 # unknown
        res = _drain(s, list(tickets))
    assert res[tickets[0]] == "ECANCELED" and res[tickets[2]] == "ECANCELED"
    np.testing.assert_array_equal(res[tickets[1]]["hubs"], alone[1]["hubs"])
    assert res[tickets[1]]["cost_fp64"] == alone[1]["cost_fp64"]


@pytest.mark.parametrize("path", [PATH_PLAIN_FP32, PATH_SPLIT_BF16], ids=["plain", "split"])
def test_resumed_run_equals_uninterrupted_run(path):
    inst = synth.urand200(seed=9, n=140, p=7)
    prm = dict(islands=3, island_size=16, n1=4, path=path)
    with Instance.from_instance(inst) as gi:
        gi.set_params(**prm)
        gi.ga_begin(77)
        gi.ga_run(21)
        whole = gi.ga_result()
        m_whole, f_whole = gi.ga_islands()
    with Instance.from_instance(inst) as gi:
        gi.set_params(**prm)
        gi.ga_begin(77)
        gi.ga_run(9)
        state = gi.ga_save()
    with Instance.from_instance(inst) as gi:
        gi.set_params(**prm)
        gi.ga_load(state)
        gi.ga_run(12)
        resumed = gi.ga_result()
        m_res, f_res = gi.ga_islands()
        np.testing.assert_array_equal(m_res, m_whole)
        np.testing.assert_array_equal(f_res, f_whole)
    np.testing.assert_array_equal(resumed["hubs"], whole["hubs"])
    assert resumed["cost_fp64"] == whole["cost_fp64"] and resumed["cost_fp32"] == whole["cost_fp32"]
    assert resumed["evals"] == whole["evals"]


def test_states_from_other_parameters_are_refused():
    inst = synth.urand200(seed=10, n=60, p=5)
    with Instance.from_instance(inst) as gi:
        gi.set_params(islands=2, island_size=8)
        gi.ga_begin(1)
        gi.ga_run(3)
        state = gi.ga_save()
        gi.set_params(islands=4)
        with pytest.raises(UsaphmpError):
            gi.ga_load(state)                              # another size
        gi.set_params(islands=2, n1=5)
        with pytest.raises(UsaphmpError):
            gi.ga_load(state)                              # same size, other n1
        gi.set_params(n1=10)
        bad = bytearray(state)
        bad[0] ^= 0xFF
        with pytest.raises(UsaphmpError):
            gi.ga_load(bytes(bad))                         # not a state
        gi.ga_load(state)
        gi.ga_run(1)


def test_destroyed_handles_give_back_their_device_memory():
    """A handle that ran every kind of work (GA, batch local search with its
    kept scratch, rescoring, evaluation) returns all its device memory when it
    is destroyed: the device's free memory after three create/run/destroy
    cycles equals that after the first (which also loads the kernels)."""
    import torch
    from gpu_util import dev, stream
    inst = synth.clustered(seed=17, n=600, p=20)
    B, ns = 64, 640
    hubs, S = synth.random_population(18, inst.n, inst.p, B)
    hs = np.sort(hubs, axis=1).astype(np.int32)
    d_hs = dev(hs)
    d_slot = torch.empty((B, ns), dtype=torch.uint8, device="cuda")
    d_cost = torch.empty(B, dtype=torch.float64, device="cuda")

    def cycle():
        with Instance.from_instance(inst) as gi:
            assert gi.ns == ns
            gi.set_params(islands=4, island_size=16)
            gi.solve(3, 1)
            gi.allocate_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), stream())
            gi.local_search_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), 3)
            gi.rescore_fp64_dev(B, d_hs.data_ptr(), d_slot.data_ptr(), d_cost.data_ptr(), stream())
            assert np.isfinite(gi.eval(hubs, S)).all()
        torch.cuda.synchronize()

    cycle()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    # the local-search scratch alone is B*(2np + p(p|1)) doubles = 12.5 MB per handle here
    assert free1 >= free0 - (2 << 20), (free0 - free1) / 2**20
